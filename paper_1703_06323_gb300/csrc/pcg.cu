// BDDC-preconditioned CG on the device (Sect. 5.1 stopping rule |r| < rtol |b|).
//
// A solve is one instantiated CUDA graph: the initial residual and preconditioner,
// then a conditional while node whose body is one iteration (the body's last kernel
// decides whether to run again, from the device-side convergence state), then the
// true residual.  The host launches it once and reads the result once; nothing
// returns to the host between iterations.  One iteration is six kernels (seven
// with the coarse prolongation):
//   K1  p = z + beta p (double-buffered, computed once per node of a tile with its
//       halo) and q = A p, element by element; partial p.q
//   K2  alpha = r.z / p.q;  x += alpha p;  r -= alpha q;  |r|^2, convergence
//   K3  per subdomain: y_I = A_II^-1 r_I, t_G = A_GI y_I          (Eq. bddc, first term
//       and E^T = I - A I0 A0^-1 I0^T)
//   K4  per subdomain: r~_G = w (r_G - sum_w' t_G^w') (weighted restriction W^T E^T r),
//       v = K r~ (constrained Neumann), g = Phi^T r~ (coarse residual part)
//   K5  coarse: r_c = sum R_c^T g, u_c = A_c^-1 r_c
//   K7  per subdomain: u_G = sum_w' w' (v + Phi u_c) (weighting W), z_G = u_G,
//       z_I = A_II^-1 (r_I - A_IG u_G) (harmonic extension); partial r.z
// Scalars live on the device.  Reductions are done by the last CTA to finish
// (fixed summation order, deterministic).
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include <cooperative_groups.h>

#include "bddc.cuh"
#include "q1.cuh"

namespace ufe {

namespace cg = cooperative_groups;

constexpr int kApplyThreads = 256;
constexpr int kSubThreads = 256;
constexpr int kCL = 4;   // CTAs (one thread-block cluster) per subdomain in the preconditioner stages

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// a warp sum in the operator's precision: FP32 partials of the FP32 operators are
// summed in FP32 (five FP64 adds per row cost more FP64-pipe time on this part than
// the whole FP32 row product), FP64 ones in FP64
__device__ __forceinline__ float warp_sum_tm(float v) { return warp_sumf(v); }
__device__ __forceinline__ double warp_sum_tm(double v) { return warp_sum(v); }

// deterministic block sum (fixed tree); all threads get the result
__device__ double block_sum(double v) {
  __shared__ double ws[32];
  __shared__ double tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < nw ? ws[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) tot = t;
  }
  __syncthreads();
  const double r = tot;
  __syncthreads();
  return r;
}

// true in exactly one CTA: the last one to arrive (after all partials are visible)
__device__ bool arrive_last(unsigned int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicInc(counter, gridDim.x - 1) == gridDim.x - 1;
  __syncthreads();
  return last;
}

// sum of part[0..n) in a fixed order (called by one whole CTA)
__device__ double sum_partials(const double* part, int n, int stride) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[(int64_t)i * stride];
  return block_sum(v);
}

// ---------------------------------------------------------------------------
// element-by-element operator apply (Sect. 2.2): internal cells use kappa h Khat,
// cut cells their own 8x8 matrix
struct OpArgs {
  GridGeom g;
  int64_t n_dof;            // free nodes
  const int32_t* node_of_dof;
  const int32_t* dof_of_node;
  const uint8_t* cell_type;
  const int32_t* cut_index;
  const double* K_cut;      // n_cut x (8 ncomp)^2
  const double* kappa;
  const double* Kref;       // elasticity: h Khat_el
  const int32_t* tiles;     // node tiles holding a free DOF (one CTA each)
  int64_t n_tiles;
};

// The operator is applied on node tiles: one CTA per kTX x kTY x kTZ box of grid nodes
// (one thread per node), with the box's input values and a one-node halo
// (kHX x kHY x kHZ), the DOF numbers of those nodes and the kCX x kCY x kCZ cells
// around the box staged in shared memory.  Every input value and cell record is then
// read from global memory once per tile instead of once per neighbouring row.
constexpr int kTX = kApplyTX, kTY = kApplyTY, kTZ = kApplyTZ;
constexpr int kTileThreads = kTX * kTY * kTZ;
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHZ = kTZ + 2, kHalo = kHX * kHY * kHZ;
constexpr int kCX = kTX + 1, kCY = kTY + 1, kCZ = kTZ + 1, kTileCells = kCX * kCY * kCZ;
constexpr int kHaloPer = (kHalo + kTileThreads - 1) / kTileThreads;
constexpr int kCellsPer = (kTileCells + kTileThreads - 1) / kTileThreads;
constexpr int32_t kCellInternal = -1, kCellNone = -2;

template <int NC>
struct ApplyTile {
  double x[NC][kHalo];
  double kap[kTileCells];
  int32_t code[kTileCells];   // cut index, kCellInternal, or kCellNone (external / off the grid)
  int32_t dof[kHalo];
  int16_t node[kTileThreads];  // the box's free nodes, in box order (thread t takes node[t])
  int32_t warp_free[kTileThreads / 32];
};

// Stages the tile and returns the free DOF of the node the calling thread computes
// (-1 if it has none), with its NC rows of A x in y (x entry e = NC dof + component is
// load(e)) and its halo index in *hc_out.  The cells around a node are visited in the
// same order, and each cell's row summed in the same order, for every node, so results
// do not depend on the tiling.  Every thread of the CTA must call it.  The staging loads are issued in rounds
// (all DOF numbers and cell records, then all input values) so that each thread has
// all of its loads of a round in flight at once.
template <int NC, typename Load>
__device__ __forceinline__ int32_t tile_apply(const OpArgs& a, ApplyTile<NC>& T, Load load, double y[NC],
                                              int* hc_out) {
  const GridGeom& g = a.g;
  const int ntx = apply_tiles_x(g), nty = apply_tiles_y(g);
  const int t = a.tiles[blockIdx.x];
  const int x0 = (t % ntx) * kTX, y0 = ((t / ntx) % nty) * kTY, z0 = (t / (ntx * nty)) * kTZ;
  int32_t e[kHaloPer];
#pragma unroll
  for (int u = 0; u < kHaloPer; ++u) {
    const int h = (int)threadIdx.x + u * kTileThreads;
    const int i = x0 - 1 + h % kHX, j = y0 - 1 + (h / kHX) % kHY, k = z0 - 1 + h / (kHX * kHY);
    e[u] = -1;
    if (h < kHalo && i >= 0 && j >= 0 && k >= 0 && i <= g.nx && j <= g.ny && k <= g.nz)
      e[u] = a.dof_of_node[g.node(i, j, k)];
  }
  uint8_t ty[kCellsPer];
  int32_t ci[kCellsPer];
  double kp[kCellsPer];
#pragma unroll
  for (int u = 0; u < kCellsPer; ++u) {
    const int q = (int)threadIdx.x + u * kTileThreads;
    const int i = x0 - 1 + q % kCX, j = y0 - 1 + (q / kCX) % kCY, k = z0 - 1 + q / (kCX * kCY);
    ty[u] = UFE_CELL_EXTERNAL;
    ci[u] = 0;
    kp[u] = 0.0;
    if (q < kTileCells && i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz) {
      const int64_t c = g.cell(i, j, k);
      ty[u] = a.cell_type[c];
      ci[u] = a.cut_index[c];
      kp[u] = a.kappa ? a.kappa[c] : 1.0;
    }
  }
  double xv[kHaloPer][NC];
#pragma unroll
  for (int u = 0; u < kHaloPer; ++u)
#pragma unroll
    for (int c = 0; c < NC; ++c) xv[u][c] = e[u] >= 0 ? load((int64_t)NC * e[u] + c) : 0.0;
#pragma unroll
  for (int u = 0; u < kHaloPer; ++u) {
    const int h = (int)threadIdx.x + u * kTileThreads;
    if (h < kHalo) {
      T.dof[h] = e[u];
#pragma unroll
      for (int c = 0; c < NC; ++c) T.x[c][h] = xv[u][c];
    }
  }
#pragma unroll
  for (int u = 0; u < kCellsPer; ++u) {
    const int q = (int)threadIdx.x + u * kTileThreads;
    if (q < kTileCells) {
      T.code[q] = ty[u] == UFE_CELL_EXTERNAL ? kCellNone : (ty[u] == UFE_CELL_INTERNAL ? kCellInternal : ci[u]);
      T.kap[q] = kp[u];
    }
  }
  __syncthreads();
  // the free nodes of the box are packed onto the first threads (most boxes are
  // partly outside the domain; the FP64 rows then run on full warps)
  {
    const int tlx = threadIdx.x % kTX, tly = (threadIdx.x / kTX) % kTY, tlz = threadIdx.x / (kTX * kTY);
    const bool free_node = T.dof[(tlx + 1) + kHX * ((tly + 1) + kHY * (tlz + 1))] >= 0;
    const unsigned m = __ballot_sync(0xffffffffu, free_node);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) T.warp_free[wid] = __popc(m);
    __syncthreads();
    int rank = __popc(m & ((1u << lane) - 1u));
    for (int q = 0; q < wid; ++q) rank += T.warp_free[q];
    if (free_node) T.node[rank] = (int16_t)threadIdx.x;
    __syncthreads();
    int total = 0;
    for (int q = 0; q < kTileThreads / 32; ++q) total += T.warp_free[q];
    if ((int)threadIdx.x >= total) {
      *hc_out = 0;
      return -1;
    }
  }
  const int tn = T.node[threadIdx.x];
  const int lx = tn % kTX, ly = (tn / kTX) % kTY, lz = tn / (kTX * kTY);
  const int hc = (lx + 1) + kHX * ((ly + 1) + kHY * (lz + 1));
  *hc_out = hc;
  const int32_t d = T.dof[hc];
#pragma unroll
  for (int c = 0; c < NC; ++c) y[c] = 0.0;
  if constexpr (NC == 1) {
    // a node whose eight cells are all internal with one coefficient: the assembled
    // Q1 stencil, kappa h (8/3 x_0 - 1/6 sum of the 12 edge neighbours - 1/12 sum of the
    // 8 corner neighbours) (the face neighbours' entries cancel to zero)
    bool plain = true;
    const double k0 = T.kap[lx + kCX * (ly + kCY * lz)];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int cq = (lx + (q & 1)) + kCX * ((ly + ((q >> 1) & 1)) + kCY * (lz + (q >> 2)));
      plain = plain && T.code[cq] == kCellInternal && T.kap[cq] == k0;
    }
    if (plain) {
      double se = 0.0, sc = 0.0;
#pragma unroll
      for (int oz = -1; oz <= 1; ++oz)
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
          for (int ox = -1; ox <= 1; ++ox) {
            const int nz = (ox != 0) + (oy != 0) + (oz != 0);
            const double v = T.x[0][hc + ox + kHX * (oy + kHY * oz)];
            if (nz == 2) se += v;
            if (nz == 3) sc += v;
          }
      y[0] = k0 * g.h * ((8.0 / 3.0) * T.x[0][hc] - (1.0 / 6.0) * se - (1.0 / 12.0) * sc);
      return d;
    }
  }
#pragma unroll
  for (int dk = -1; dk <= 0; ++dk)
#pragma unroll
    for (int dj = -1; dj <= 0; ++dj)
#pragma unroll
      for (int di = -1; di <= 0; ++di) {
        // cell (lx + di, ly + dj, lz + dk) relative to the box; its vertex b sits at halo
        // offset (lx + di + 1 + (b & 1), ...)
        const int cq = (lx + di + 1) + kCX * ((ly + dj + 1) + kCY * (lz + dk + 1));
        const int32_t code = T.code[cq];
        if (code == kCellNone) continue;
        const int av = (-di) + 2 * (-dj) + 4 * (-dk);
        const double kap = T.kap[cq];
        const int h0 = (lx + di + 1) + kHX * ((ly + dj + 1) + kHY * (lz + dk + 1));
        if constexpr (NC == 1) {
          double s = 0.0;
          if (code == kCellInternal) {
#pragma unroll
            for (int b = 0; b < 8; ++b)
              s += q1_khat(av, b) * T.x[0][h0 + (b & 1) + kHX * (((b >> 1) & 1) + kHY * (b >> 2))];
            s *= g.h;
          } else {
            const double* Kc = a.K_cut + (int64_t)code * 64 + av * 8;
#pragma unroll
            for (int b = 0; b < 8; ++b) s += Kc[b] * T.x[0][h0 + (b & 1) + kHX * (((b >> 1) & 1) + kHY * (b >> 2))];
          }
          y[0] += kap * s;
        } else {
          // elasticity: y_c += kappa_e sum_b sum_j K_e[3 av + c][3 b + j] x_{3 e_b + j}
          const double* Ke = (code == kCellInternal ? a.Kref : a.K_cut + (int64_t)code * 576) + 3 * av * 24;
          double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            const int hb = h0 + (b & 1) + kHX * (((b >> 1) & 1) + kHY * (b >> 2));
            if (T.dof[hb] < 0) continue;
#pragma unroll
            for (int jc = 0; jc < 3; ++jc) {
              const double x = T.x[jc][hb];
              s0 += Ke[3 * b + jc] * x;
              s1 += Ke[24 + 3 * b + jc] * x;
              s2 += Ke[48 + 3 * b + jc] * x;
            }
          }
          y[0] += kap * s0;
          y[1] += kap * s1;
          y[2] += kap * s2;
        }
      }
  return d;
}

template <int NC>
__global__ void __launch_bounds__(kTileThreads) k_apply(OpArgs a, const double* __restrict__ x, double* __restrict__ y) {
  __shared__ ApplyTile<NC> T;
  double yy[NC];
  int hc;
  const int32_t d = tile_apply<NC>(a, T, [&](int64_t e) { return x[e]; }, yy, &hc);
  if (d < 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) y[NC * (int64_t)d + c] = yy[c];
}

// r = b - A x, |r|^2 and |b|^2; mode 0 initialises the scalars, mode 1 only reports |b - A x|^2
template <int NC>
__global__ void __launch_bounds__(kTileThreads)
k_residual(OpArgs a, const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ r,
           double* __restrict__ part, PcgScalars* sc, int mode, double* out) {
  __shared__ ApplyTile<NC> T;
  double ax[NC];
  int hc;
  const int32_t d = tile_apply<NC>(a, T, [&](int64_t e) { return x[e]; }, ax, &hc);
  double rr = 0.0, bb = 0.0;
  if (d >= 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int64_t e = NC * (int64_t)d + c;
      const double res = b[e] - ax[c];
      if (r) r[e] = res;
      rr += res * res;
      bb += b[e] * b[e];
    }
  }
  rr = block_sum(rr);
  bb = block_sum(bb);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rr;
    part[2 * blockIdx.x + 1] = bb;
  }
  if (arrive_last(&sc->counter[0])) {
    const double R = sum_partials(part, gridDim.x, 2);
    const double B = sum_partials(part + 1, gridDim.x, 2);
    if (threadIdx.x == 0) {
      if (mode == 0) {
        sc->rr = R;
        sc->bb = B;
        sc->tol2 = sc->rtol * sc->rtol * B;
        sc->iter = 0;
        sc->first = 1;
        sc->done = (R < sc->tol2 || B == 0.0) ? 1 : 0;
      } else {
        out[0] = R;
        out[1] = B;
      }
    }
  }
}

// K1: p_new = z + beta p_old (beta = 0 for the first direction); q = A p_new; p.q
template <int NC>
__global__ void __launch_bounds__(kTileThreads)
k_dir_apply(OpArgs a, const double* __restrict__ z, double* p0, double* p1, double* __restrict__ q,
            double* __restrict__ part, PcgScalars* sc) {
  if (sc->done) return;
  __shared__ ApplyTile<NC> T;
  const int it = sc->iter;
  const double* pold = (it & 1) ? p1 : p0;
  double* pnew = (it & 1) ? p0 : p1;
  double beta = 0.0;
  if (!sc->first) beta = sc->flexible ? (sc->rz_next - sc->rzold_next) / sc->rz : sc->rz_next / sc->rz;
  double qd[NC];
  int hc;
  const int32_t d = tile_apply<NC>(a, T, [&](int64_t e) { return z[e] + beta * pold[e]; }, qd, &hc);
  double pq = 0.0;
  if (d >= 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int64_t e = NC * (int64_t)d + c;
      const double pd = T.x[c][hc];
      pnew[e] = pd;
      q[e] = qd[c];
      pq += pd * qd[c];
    }
  }
  pq = block_sum(pq);
  if (threadIdx.x == 0) part[blockIdx.x] = pq;
  if (arrive_last(&sc->counter[1])) {
    const double P = sum_partials(part, gridDim.x, 1);
    if (threadIdx.x == 0) sc->pq = P;
  }
}

// K2: x += alpha p, r -= alpha q, |r|^2, convergence test
__global__ void __launch_bounds__(kApplyThreads)
k_update(int64_t n, double* __restrict__ x, double* __restrict__ r, const double* p0, const double* p1,
         const double* __restrict__ q, double* __restrict__ part, PcgScalars* sc) {
  if (sc->done) return;
  const int it = sc->iter;
  const double* p = (it & 1) ? p0 : p1;
  const double pq = sc->pq;
  const bool ok = pq > 0.0;
  const double alpha = ok ? sc->rz_next / pq : 0.0;
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double rr = 0.0;
  if (d < n && ok) {
    x[d] += alpha * p[d];
    const double rd = r[d] - alpha * q[d];
    r[d] = rd;
    rr = rd * rd;
  }
  rr = block_sum(rr);
  if (threadIdx.x == 0) part[blockIdx.x] = rr;
  if (arrive_last(&sc->counter[2])) {
    const double R = sum_partials(part, gridDim.x, 1);
    if (threadIdx.x == 0) {
      if (!ok) {
        sc->done = 3;
      } else {
        sc->rr = R;
        sc->iter = it + 1;
        sc->rz = sc->rz_next;
        sc->first = 0;
        if (R < sc->tol2)
          sc->done = 1;
        else if (it + 1 >= sc->maxit)
          sc->done = 2;
      }
    }
  }
}

// the condition of the device-side loop: run another iteration while the solve is
// running; every pass is counted and the loop stops after maxit + 1 passes whatever
// the state says, so it always ends
__global__ void k_loop_cond(cudaGraphConditionalHandle h, PcgScalars* sc) {
  const unsigned pass = sc->passes;
  sc->passes = pass + 1;
  const bool more = sc->done == 0 && sc->iter < sc->maxit && pass < (unsigned)sc->maxit + 1u;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// preconditioner stages
// ---------------------------------------------------------------------------
template <typename TM>
struct VecT;
template <>
struct VecT<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct VecT<double> {
  using type = double2;
  static constexpr int n = 2;
};

__device__ __forceinline__ float dot_vec(const float4& a, const float* x) {
  return a.x * x[0] + a.y * x[1] + a.z * x[2] + a.w * x[3];
}
__device__ __forceinline__ double dot_vec(const double2& a, const double* x) { return a.x * x[0] + a.y * x[1]; }

// ys[r] = sum_c M[r, c] xs[c] for r in [r0, r1) (row-major, ld a multiple of 4, xs
// zero-padded to ld); each warp streams two rows at a time with 16-byte loads
template <typename TM>
__device__ void cta_gemv_rows(const TM* __restrict__ M, int r0, int r1, int ld, const TM* __restrict__ xs,
                              double* __restrict__ ys) {
  using V = typename VecT<TM>::type;
  constexpr int VN = VecT<TM>::n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int r = r0 + wid;
  for (; r + nw < r1; r += 2 * nw) {
    const TM* ra = M + (int64_t)r * ld;
    const TM* rb = M + (int64_t)(r + nw) * ld;
    TM sa = TM(0), sb = TM(0);
    for (int c = lane * VN; c < ld; c += 32 * VN) {
      const V va = *reinterpret_cast<const V*>(ra + c);
      const V vb = *reinterpret_cast<const V*>(rb + c);
      sa += dot_vec(va, xs + c);
      sb += dot_vec(vb, xs + c);
    }
    const double da = (double)warp_sum_tm(sa), db = (double)warp_sum_tm(sb);
    if (lane == 0) {
      ys[r] = da;
      ys[r + nw] = db;
    }
  }
  for (; r < r1; r += nw) {
    const TM* ra = M + (int64_t)r * ld;
    TM sa = TM(0);
    for (int c = lane * VN; c < ld; c += 32 * VN) sa += dot_vec(*reinterpret_cast<const V*>(ra + c), xs + c);
    const double da = (double)warp_sum_tm(sa);
    if (lane == 0) ys[r] = da;
  }
}

// launch parameters shared by the per-subdomain kernels
struct SubLaunch {
  int ldImax, ldGmax;   // largest padded interior / interface sizes
  int n_stages;         // row-stream stages per CTA (1..kMaxStages)
  int stream_rows;      // rows per stage (kStreamRows, or fewer when one stage of long rows would not fit)
  // the subdomains of this launch: wl[cluster] (null: cluster c is subdomain c); with
  // subdomains in two precisions each stage is two launches, and the final stage's
  // dot products are partials part_off + CTA, summed (n_final of them) only by the
  // last CTA of the launch with n_final > 0
  const int32_t* wl;
  int part_off, n_final;
};

// the subdomain of this CTA's cluster
template <int CL>
__device__ __forceinline__ int sub_of_cluster(const SubLaunch& L) {
  const int c = (int)blockIdx.x / CL;
  return L.wl ? L.wl[c] : c;
}

struct SubSizes {
  int nI, nG, nC, ldI, ldG, ldC, bi, bj, bk;
};
__device__ __forceinline__ SubSizes sub_sizes(const SubMeta& sm, int w) {
  SubSizes z;
  z.nI = sm.vI_ptr[w + 1] - sm.vI_ptr[w];
  z.nG = sm.vG_ptr[w + 1] - sm.vG_ptr[w];
  z.nC = sm.C_ptr[w + 1] - sm.C_ptr[w];
  z.ldI = pad4(z.nI);
  z.ldG = pad4(z.nG);
  z.ldC = pad4(z.nC);
  const int b = sm.sub_block[w];
  z.bi = b % sm.g.bx;
  z.bj = (b / sm.g.bx) % sm.g.by;
  z.bk = b / (sm.g.bx * sm.g.by);
  return z;
}

// global vector DOF of local interior vector index p of subdomain w
template <int NC>
__device__ __forceinline__ int64_t vdof_I(const SubMeta& sm, int w, int p) {
  return (int64_t)NC * sm.I_list[sm.I_ptr[w] + p / NC] + p % NC;
}

// shared memory layout shared by the per-subdomain kernels
struct SubSmem {
  double* dI;     // ldImax doubles
  double* dG;     // ldGmax doubles
  void* xT;       // max(ldImax, ldGmax) TM values
  void* stage;    // row-stream stages (128-byte aligned)
};

__device__ __forceinline__ SubSmem carve(char* smem, int ldImax, int ldGmax, size_t tm_size) {
  SubSmem s;
  size_t off = 0;
  s.dI = reinterpret_cast<double*>(smem + off);
  off += (size_t)ldImax * 8;
  s.dG = reinterpret_cast<double*>(smem + off);
  off += (size_t)ldGmax * 8;
  s.xT = smem + off;
  off += (size_t)(ldImax > ldGmax ? ldImax : ldGmax) * tm_size;
  off = (off + 127) & ~(size_t)127;
  s.stage = smem + off;
  return s;
}

// ---------------------------------------------------------------------------
// row streaming: the rows of a CTA's slice of a dense local operator are moved
// from HBM into a ring of shared-memory stages by bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier), kStreamRows rows per stage
// (fewer for rows too long to fit eight in shared memory: 16-cell blocks in FP64),
// so that a whole stage per CTA is in flight while the previous one is consumed.
// One warp per row of a stage (with R < kStreamRows rows, kStreamRows / R warps split
// each row's columns and their sums are added in warp order); each lane reads 16
// bytes at a time from shared memory.  Every wait is bounded by a wall-clock limit; on expiry the CTA records
// DEV_TIMEOUT, drains its copies (again bounded) and leaves its results undefined.
// ---------------------------------------------------------------------------
constexpr int kStreamRows = kSubThreads / 32;
constexpr int kMaxStages = 4;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // one second

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity; false after the limit
__device__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

template <typename TM>
struct RowStream {
  const TM* M;      // first row of the slice
  TM* buf;          // n_stages * R * ld values
  uint64_t* full;   // one barrier per stage
  double* part;     // kStreamRows partial row sums (R < kStreamRows)
  int rows, ld, n_stages, n_steps, R;

  __device__ void issue(int step) const {
    const int row0 = step * R;
    const int nr = min(R, rows - row0);
    const int slot = step % n_stages;
    const unsigned bytes = (unsigned)(nr * ld * (int)sizeof(TM));
    mbar_arrive_tx(&full[slot], bytes);
    bulk_load(buf + (size_t)slot * R * ld, M + (size_t)row0 * ld, bytes, &full[slot]);
  }
  // thread 0: initialise the barriers and put the first stages in flight; the
  // other threads may wait on them only after a later __syncthreads
  __device__ void begin(const TM* M_, int r0, int r1, int ld_, void* stage, uint64_t* bars, double* part_,
                        const SubLaunch& L) {
    M = M_ + (size_t)r0 * ld_;
    buf = reinterpret_cast<TM*>(stage);
    full = bars;
    part = part_;
    rows = r1 - r0;
    ld = ld_;
    n_stages = L.n_stages;
    R = L.stream_rows;
    n_steps = (rows + R - 1) / R;
    if (threadIdx.x == 0) {
      for (int i = 0; i < n_stages; ++i) mbar_init(&full[i], 1);
      mbar_fence_init();
      for (int i = 0; i < min(n_stages, n_steps); ++i) issue(i);
    }
  }
  // ys[r0 + i] = sum_c M[r0 + i, c] xs[c] (xs zero-padded to ld, in shared memory)
  __device__ void gemv(const TM* __restrict__ xs, double* __restrict__ ys, int* status) const {
    using V = typename VecT<TM>::type;
    constexpr int VN = VecT<TM>::n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int step = 0; step < n_steps; ++step) {
      const int slot = step % n_stages;
      const bool ok = mbar_wait(&full[slot], (unsigned)((step / n_stages) & 1));
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          atomicOr(status, DEV_TIMEOUT);
          for (int s2 = step; s2 < min(step + n_stages, n_steps); ++s2)
            mbar_wait(&full[s2 % n_stages], (unsigned)((s2 / n_stages) & 1));
        }
        __syncthreads();
        return;
      }
      if (R == kStreamRows) {
        const int i = step * kStreamRows + wid;
        if (i < rows) {
          const TM* row = buf + ((size_t)slot * kStreamRows + wid) * ld;
          TM acc = TM(0);
          for (int c = lane * VN; c < ld; c += 32 * VN) acc += dot_vec(*reinterpret_cast<const V*>(row + c), xs + c);
          const double d = (double)warp_sum_tm(acc);
          if (lane == 0) ys[i] = d;
        }
        __syncthreads();
      } else {
        // P = kStreamRows / R warps per row, each over every P-th chunk of 32 VN columns
        const int P = kStreamRows / R, rl = wid / P, q = wid % P;
        const int i = step * R + rl;
        if (i < rows) {
          const TM* row = buf + ((size_t)slot * R + rl) * ld;
          TM acc = TM(0);
          for (int c = (q * 32 + lane) * VN; c < ld; c += 32 * VN * P)
            acc += dot_vec(*reinterpret_cast<const V*>(row + c), xs + c);
          const double d = (double)warp_sum_tm(acc);
          if (lane == 0) part[wid] = d;
        }
        __syncthreads();
        if ((int)threadIdx.x < R && step * R + (int)threadIdx.x < rows) {
          double d = 0.0;
          for (int x = 0; x < P; ++x) d += part[threadIdx.x * P + x];
          ys[step * R + threadIdx.x] = d;
        }
      }
      if (threadIdx.x == 0 && step + n_stages < n_steps) issue(step + n_stages);
    }
    if (R != kStreamRows) __syncthreads();   // the last step's sums are written after its barrier
  }
};

// ys[r] = sum_c M[r, c] xs[c] for short rows (ld <= 32 * VN): groups of G lanes per row
template <typename TM>
__device__ void cta_gemv_short(const TM* __restrict__ M, int r0, int r1, int ld, const TM* __restrict__ xs,
                               double* __restrict__ ys) {
  using V = typename VecT<TM>::type;
  constexpr int VN = VecT<TM>::n;
  int G = 1;
  while (G * VN < ld && G < 32) G <<= 1;
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  const int per_warp = 32 / G;
  const int gid = (threadIdx.x >> 5) * per_warp + lane / G, ng = (blockDim.x >> 5) * per_warp;
  for (int rb = r0; rb < r1; rb += ng) {
    const int r = rb + gid;
    TM acc = TM(0);
    if (r < r1) {
      const TM* row = M + (int64_t)r * ld;
      for (int c = sub * VN; c < ld; c += G * VN) acc += dot_vec(*reinterpret_cast<const V*>(row + c), xs + c);
    }
    TM d = acc;
    for (int o = G >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (r < r1 && sub == 0) ys[r] = (double)d;
  }
}

// The per-subdomain stages run as thread-block clusters of CL CTAs per subdomain (2, 4
// or 8, chosen per problem by the launch-shape tuner): each CTA computes a contiguous
// slice of the rows of a local GEMV and the slices are exchanged through distributed
// shared memory.
template <int CL>
__device__ __forceinline__ void row_slice(int n, int rank, int& b, int& e) {
  b = (n * rank) / CL;
  e = (n * (rank + 1)) / CL;
}

// copy the slices of `local` that the other CTAs of the cluster computed
template <int CL, typename V>
__device__ void cluster_gather(cg::cluster_group& cl, V* local, int n) {
  const int me = (int)cl.block_rank();
  for (int r = 0; r < CL; ++r) {
    if (r == me) continue;
    int b, e;
    row_slice<CL>(n, r, b, e);
    const V* remote = cl.map_shared_rank(local, r);
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) local[i] = remote[i];
  }
}

// acc + sign v[NC s_k + c] for the first cnt slots s_k = gpos[8 xi + k] of node xi, added
// in slot order; the eight slots and then the values are loaded together
template <int NC>
__device__ __forceinline__ double gather_slots(const int32_t* __restrict__ gpos, int64_t xi, int cnt, int c,
                                              const double* __restrict__ v, double acc, double sign) {
  const int4 pa = *reinterpret_cast<const int4*>(gpos + xi * 8);
  const int4 pb = *reinterpret_cast<const int4*>(gpos + xi * 8 + 4);
  const int sl[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = k < cnt ? v[(int64_t)NC * sl[k] + c] : 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (k < cnt) acc += sign * x[k];
  return acc;
}

// K3: y_I = A_II^-1 r_I; t_G = A_GI y_I
template <typename TM, int NC, int CL = kCL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kSubThreads)
k_prec_interior1(SubMeta sm, const TM* __restrict__ AIIinv, const double* __restrict__ r, double* __restrict__ tG,
                 const PcgScalars* sc, SubLaunch L) {
  if (sc && sc->done) return;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) char smem[];
  const int w = sub_of_cluster<CL>(L), rank = (int)cl.block_rank();
  const SubSizes z = sub_sizes(sm, w);
  SubSmem S = carve(smem, L.ldImax, L.ldGmax, sizeof(TM));
  __shared__ uint64_t full[kMaxStages];
  __shared__ double rpart[kStreamRows];
  int r0, r1;
  row_slice<CL>(z.nI, rank, r0, r1);
  RowStream<TM> rs;
  rs.begin(AIIinv + sm.off_II[w], r0, r1, z.ldI, S.stage, full, rpart, L);
  TM* xI = reinterpret_cast<TM*>(S.xT);
  const int i0 = sm.vI_ptr[w];
  for (int p = threadIdx.x; p < z.ldI; p += blockDim.x)
    xI[p] = p < z.nI ? (TM)(sm.sI[i0 + p] * r[vdof_I<NC>(sm, w, p)]) : TM(0);
  __syncthreads();
  rs.gemv(xI, S.dI + r0, sm.status);
  cl.sync();
  cluster_gather<CL>(cl, S.dI, z.nI);
  cl.sync();
  // y_I = S_I (Ahat_II^-1 (S_I r_I)), on every CTA's full copy
  for (int p = threadIdx.x; p < z.nI; p += blockDim.x) S.dI[p] *= sm.sI[i0 + p];
  __syncthreads();
  int j0, j1;
  row_slice<CL>(z.nG, rank, j0, j1);
  constexpr int KS = 27 * NC;
  const int64_t e0 = KS * (int64_t)sm.vG_ptr[w];
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    double t = 0.0;
#pragma unroll 27
    for (int o = 0; o < KS; ++o) {
      const int32_t k = sm.gi_k[e0 + (int64_t)o * z.nG + j];
      if (k >= 0) t += sm.gi_v[e0 + (int64_t)o * z.nG + j] * S.dI[k];
    }
    tG[sm.vG_ptr[w] + j] = t;
  }
}

// one term of a compensated FP32 dot product (Ogita, Rump, Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26 (2005), Dot2): a + e accumulates p (x + l);
// the rounded intrinsics keep the compiler from fusing the product into the sum
__device__ __forceinline__ void dot2_step(float& a, float& e, float p, float x, float l) {
  const float prod = __fmul_rn(p, x);
  const float perr = fmaf(p, x, -prod);
  const float s = __fadd_rn(a, prod);
  const float bp = __fsub_rn(s, a);
  const float serr = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(prod, bp));
  a = s;
  e = fmaf(p, l, e + serr + perr);
}
__device__ __forceinline__ void dot2_step(double&, double&, double, double, double) {}

// K4: r~ = w (r_G - sum t_G); v = K r~ (stored weighted: vw = w v); g = Phi^T r~
template <typename TM, int NC, int CL = kCL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kSubThreads)
k_prec_neumann(SubMeta sm, const TM* __restrict__ Kop, const TM* __restrict__ Phi, const double* __restrict__ r,
               const double* __restrict__ tG, double* __restrict__ vw, double* __restrict__ gC, const PcgScalars* sc,
               SubLaunch L) {
  if (sc && sc->done) return;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) char smem[];
  __shared__ double gpart[kSubThreads / 32][64];
  __shared__ double gsum[1024];
  const int w = sub_of_cluster<CL>(L), rank = (int)cl.block_rank();
  const SubSizes z = sub_sizes(sm, w);
  if (z.nG == 0) return;
  SubSmem S = carve(smem, L.ldImax, L.ldGmax, sizeof(TM));
  __shared__ uint64_t full[kMaxStages];
  __shared__ double rpart[kStreamRows];
  int r0, r1;
  row_slice<CL>(z.nG, rank, r0, r1);
  RowStream<TM> rs;
  rs.begin(Kop + sm.off_GG[w], r0, r1, z.ldG, S.stage, full, rpart, L);
  TM* xG = reinterpret_cast<TM*>(S.xT);
  // FP32 operators: the part of r~ below FP32 precision, kept in dG's storage until
  // the rows of K overwrite it (after the coarse restriction below has read it)
  float* xlo = reinterpret_cast<float*>(S.dG);
  const int g0 = sm.vG_ptr[w];
  for (int j = threadIdx.x; j < z.ldG; j += blockDim.x) {
    TM v = TM(0);
    double t = 0.0;
    if (j < z.nG) {
      const int32_t xi = sm.G_list[sm.G_ptr[w] + j / NC];
      const int c = j % NC;
      const double s = gather_slots<NC>(sm.gpos, xi, sm.n_neigh[xi], c, tG, r[(int64_t)NC * xi + c], -1.0);
      t = sm.sG[g0 + j] * sm.w[g0 + j] * s;
      v = (TM)t;
    }
    xG[j] = v;
    if constexpr (sizeof(TM) == 4) xlo[j] = (float)(t - (double)v);
  }
  __syncthreads();
  // partial g = Phi^T r~ over this CTA's rows (while the first rows of K are in
  // flight): warps split the rows, lanes the columns.  With FP32 operators the sums
  // are compensated (Ogita, Rump and Oishi's Dot2: the exact error of every product
  // by FMA, of every addition by Knuth's TwoSum, plus Phi times the low part of r~):
  // coarse residual parts cancel heavily next to tiny cut cells, where a plain FP32
  // sum depends on how the rows are split over CTAs
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const TM* P = Phi + sm.off_GC[w];
  for (int c0 = 0; c0 < z.nC; c0 += 64) {
    TM a0 = TM(0), a1 = TM(0), e0 = TM(0), e1 = TM(0);
#pragma unroll 4
    for (int j = r0 + wid; j < r1; j += nw) {
      const TM xj = xG[j];
      if constexpr (sizeof(TM) == 4) {
        const float lj = xlo[j];
        if (c0 + lane < z.nC) dot2_step(a0, e0, P[(int64_t)j * z.ldC + c0 + lane], xj, lj);
        if (c0 + lane + 32 < z.nC) dot2_step(a1, e1, P[(int64_t)j * z.ldC + c0 + lane + 32], xj, lj);
      } else {
        if (c0 + lane < z.nC) a0 += P[(int64_t)j * z.ldC + c0 + lane] * xj;
        if (c0 + lane + 32 < z.nC) a1 += P[(int64_t)j * z.ldC + c0 + lane + 32] * xj;
      }
    }
    gpart[wid][lane] = (double)a0 + (double)e0;
    gpart[wid][lane + 32] = (double)a1 + (double)e1;
    __syncthreads();
    if (threadIdx.x < 64 && c0 + (int)threadIdx.x < z.nC) {
      double sacc = 0.0;
      for (int x = 0; x < nw; ++x) sacc += gpart[x][threadIdx.x];
      gsum[c0 + threadIdx.x] = sacc;
    }
    __syncthreads();
  }
  rs.gemv(xG, S.dG + r0, sm.status);
  for (int j = r0 + threadIdx.x; j < r1; j += blockDim.x) vw[g0 + j] = sm.w[g0 + j] * sm.sG[g0 + j] * S.dG[j];
  cl.sync();
  if (rank == 0) {
    for (int c = threadIdx.x; c < z.nC; c += blockDim.x) {
      double sacc = 0.0;
      for (int q = 0; q < CL; ++q) sacc += cl.map_shared_rank(gsum, q)[c];
      gC[sm.C_ptr[w] + c] = sacc;
    }
  }
  cl.sync();
}

// K6: coarse prolongation, vw += w Phi u_c^w on the interface rows of w
template <typename TM, int NC, int CL = kCL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kSubThreads)
k_prec_prolong(SubMeta sm, const TM* __restrict__ Phi, const double* __restrict__ uc, double* __restrict__ vw,
               const PcgScalars* sc, SubLaunch L) {
  if (sc && sc->done) return;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) char smem[];
  const int w = sub_of_cluster<CL>(L), rank = (int)cl.block_rank();
  const SubSizes z = sub_sizes(sm, w);
  if (z.nG == 0 || z.nC == 0) return;
  SubSmem S = carve(smem, L.ldImax, L.ldGmax, sizeof(TM));
  TM* xc = reinterpret_cast<TM*>(S.xT);
  for (int c = threadIdx.x; c < z.ldC; c += blockDim.x) xc[c] = c < z.nC ? (TM)uc[sm.C_list[sm.C_ptr[w] + c]] : TM(0);
  __syncthreads();
  int j0, j1;
  row_slice<CL>(z.nG, rank, j0, j1);
  if (z.ldC <= 32 * VecT<TM>::n)
    cta_gemv_short<TM>(Phi + sm.off_GC[w], j0, j1, z.ldC, xc, S.dG);
  else
    cta_gemv_rows<TM>(Phi + sm.off_GC[w], j0, j1, z.ldC, xc, S.dG);
  __syncthreads();
  const int g0 = sm.vG_ptr[w];
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) vw[g0 + j] += sm.w[g0 + j] * sm.sG[g0 + j] * S.dG[j];
}

// K7: u_G = sum_w' w' (v + Phi u_c) (the weighted local values, W); z_G = u_G (the
// owner writes); z_I = A_II^-1 (r_I - A_IG u_G) (harmonic extension)
template <typename TM, int NC, int CL = kCL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kSubThreads)
k_prec_final(SubMeta sm, const TM* __restrict__ AIIinv, const double* __restrict__ r, const double* __restrict__ vw,
             double* __restrict__ z, double* __restrict__ part, PcgScalars* sc, SubLaunch L, int with_dots) {
  if (sc && sc->done) return;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) char smem[];
  const int w = sub_of_cluster<CL>(L), rank = (int)cl.block_rank();
  const SubSizes zz = sub_sizes(sm, w);
  SubSmem S = carve(smem, L.ldImax, L.ldGmax, sizeof(TM));
  __shared__ uint64_t full[kMaxStages];
  __shared__ double rpart[kStreamRows];
  int p0, p1;
  row_slice<CL>(zz.nI, rank, p0, p1);
  RowStream<TM> rs;
  rs.begin(AIIinv + sm.off_II[w], p0, p1, zz.ldI, S.stage, full, rpart, L);
  TM* xI = reinterpret_cast<TM*>(S.xT);
  double rz = 0.0, rzo = 0.0;
  const int gn0 = sm.G_ptr[w];
  // the whole interface vector of w (cheap gathers, computed by every CTA)
  for (int j = threadIdx.x; j < zz.nG; j += blockDim.x) {
    const int32_t xi = sm.G_list[gn0 + j / NC];
    const int c = j % NC;
    S.dG[j] = gather_slots<NC>(sm.gpos, xi, sm.n_neigh[xi], c, vw, 0.0, 1.0);
  }
  __syncthreads();
  int j0, j1;
  row_slice<CL>(zz.nG, rank, j0, j1);
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const int32_t xi = sm.G_list[gn0 + j / NC];
    if (sm.neigh[(int64_t)xi * 8] != w) continue;
    const int64_t e = (int64_t)NC * xi + j % NC;
    const double u = S.dG[j];
    if (with_dots) {
      rz += r[e] * u;
      rzo += r[e] * z[e];
    }
    z[e] = u;
  }
  // interior right-hand side r_I - A_IG u_G for this CTA's rows, then exchanged
  constexpr int KS = 27 * NC;
  const int64_t e0 = KS * (int64_t)sm.vI_ptr[w];
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    double t = 0.0;
#pragma unroll 27
    for (int o = 0; o < KS; ++o) {
      const int32_t k = sm.ig_k[e0 + (int64_t)o * zz.nI + p];
      if (k >= 0) t += sm.ig_v[e0 + (int64_t)o * zz.nI + p] * S.dG[k];
    }
    xI[p] = (TM)(sm.sI[sm.vI_ptr[w] + p] * (r[vdof_I<NC>(sm, w, p)] - t));
  }
  for (int p = zz.nI + threadIdx.x; p < zz.ldI; p += blockDim.x) xI[p] = TM(0);
  cl.sync();
  cluster_gather<CL>(cl, xI, zz.nI);
  cl.sync();
  rs.gemv(xI, S.dI + p0, sm.status);
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const int64_t d = vdof_I<NC>(sm, w, p);
    const double zn = sm.sI[sm.vI_ptr[w] + p] * S.dI[p];
    if (with_dots) {
      rz += r[d] * zn;
      rzo += r[d] * z[d];
    }
    z[d] = zn;
  }
  if (!with_dots) return;
  rz = block_sum(rz);
  rzo = block_sum(rzo);
  if (threadIdx.x == 0) {
    part[2 * (L.part_off + blockIdx.x)] = rz;
    part[2 * (L.part_off + blockIdx.x) + 1] = rzo;
  }
  if (L.n_final == 0) return;
  if (arrive_last(&sc->counter[3])) {
    const double a = sum_partials(part, L.n_final, 2);
    const double b = sum_partials(part + 1, L.n_final, 2);
    if (threadIdx.x == 0) {
      sc->rz_next = a;
      sc->rzold_next = b;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static OpArgs op_args(const System& sys) {
  const Mesh& m = *sys.mesh;
  OpArgs a;
  a.g = m.g;
  a.n_dof = m.n_dof;
  a.node_of_dof = m.node_of_dof.p;
  a.dof_of_node = m.dof_of_node.p;
  a.cell_type = m.cell_type.p;
  a.cut_index = m.cut_index.p;
  a.K_cut = sys.K_cut.p;
  a.kappa = sys.has_kappa ? sys.kappa.p : nullptr;
  a.Kref = sys.Kref.p;
  a.tiles = m.apply_tiles.p;
  a.n_tiles = m.n_apply_tiles;
  return a;
}

// adjoint contraction (no counterpart in the paper): with A = sum_e kappa_e Khat_e and
// b independent of kappa, dJ/dkappa_e = -ubar_e^T Khat_e lambda_e, where ubar holds the
// free values u and the Dirichlet values at constrained nodes and lambda vanishes there
__global__ void k_kappa_gradient(OpArgs a, const double* __restrict__ u, const double* __restrict__ lam,
                                 const double* __restrict__ gnode, double* __restrict__ out) {
  const GridGeom& g = a.g;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.n_cells()) return;
  const uint8_t t = a.cell_type[c];
  if (t == UFE_CELL_EXTERNAL) {
    out[c] = 0.0;
    return;
  }
  const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((int64_t)g.nx * g.ny));
  double ue[8], le[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const int64_t node = g.node(i + (v & 1), j + ((v >> 1) & 1), k + (v >> 2));
    const int32_t d = a.dof_of_node[node];
    ue[v] = d >= 0 ? u[d] : gnode[node];
    le[v] = d >= 0 ? lam[d] : 0.0;
  }
  const double* Kc = t == UFE_CELL_CUT ? a.K_cut + (int64_t)a.cut_index[c] * 64 : nullptr;
  double sacc = 0.0;
#pragma unroll
  for (int va = 0; va < 8; ++va) {
    double row = 0.0;
#pragma unroll
    for (int vb = 0; vb < 8; ++vb) row += (Kc ? Kc[va * 8 + vb] : g.h * q1_khat(va, vb)) * le[vb];
    sacc += ue[va] * row;
  }
  out[c] = -sacc;
}

void kappa_gradient(const System& sys, const double* u_dev, const double* lambda_dev, double* out_dev, cudaStream_t s) {
  const OpArgs a = op_args(sys);
  k_kappa_gradient<<<grid_for(a.g.n_cells(), 256), 256, 0, s>>>(a, u_dev, lambda_dev, sys.gnode.p, out_dev);
  UFE_CHECK_LAUNCH();
}

void system_apply(const System& sys, const double* x_dev, double* y_dev, cudaStream_t s) {
  const OpArgs a = op_args(sys);
  TimedLaunch t;
  t.begin("apply", s);
  if (sys.ncomp == 3)
    k_apply<3><<<(unsigned)a.n_tiles, kTileThreads, 0, s>>>(a, x_dev, y_dev);
  else
    k_apply<1><<<(unsigned)a.n_tiles, kTileThreads, 0, s>>>(a, x_dev, y_dev);
  UFE_CHECK_LAUNCH();
  t.end(s);
}

// shared-memory size and stage count of the per-subdomain kernels: the row-stream
// ring gets about 26 KB, so that five CTAs fit on an SM next to each other.  Rows so
// long that one stage of kStreamRows of them does not fit next to the vectors (FP64
// operators of 16-cell blocks) are streamed fewer to a stage.
constexpr size_t kStageBudget = 26 * 1024;
constexpr int kMaxDynSmem = 211 * 1024;

static SubLaunch sub_launch(const Bddc& B, size_t tm_size, size_t* smem) {
  SubLaunch L;
  L.ldImax = pad4(std::max(B.max_nIv, 1));
  L.ldGmax = pad4(std::max(B.max_nGv, 1));
  const size_t ldmax = (size_t)std::max(L.ldImax, L.ldGmax);
  size_t off = (size_t)L.ldImax * 8 + (size_t)L.ldGmax * 8 + ldmax * tm_size;
  off = (off + 127) & ~(size_t)127;
  L.stream_rows = kStreamRows;
  while (L.stream_rows > 1 && off + (size_t)L.stream_rows * ldmax * tm_size > (size_t)kMaxDynSmem) L.stream_rows >>= 1;
  const size_t stage = (size_t)L.stream_rows * ldmax * tm_size;
  L.n_stages = (int)std::max<size_t>(1, std::min<size_t>(kMaxStages, kStageBudget / stage));
  if (B.prec_stages > 0) L.n_stages = std::min(B.prec_stages, kMaxStages);   // tuned
  // never more stages than fit
  while (L.n_stages > 1 && off + (size_t)L.n_stages * stage > (size_t)kMaxDynSmem) --L.n_stages;
  *smem = off + (size_t)L.n_stages * stage;
  return L;
}

// the stored local operators of precision TM
template <typename TM>
struct LocalOps;
template <>
struct LocalOps<float> {
  static const float* II(const Bddc& B) { return B.fII.p; }
  static const float* GG(const Bddc& B) { return B.fGG.p; }
  static const float* GC(const Bddc& B) { return B.fGC.p; }
};
template <>
struct LocalOps<double> {
  static const double* II(const Bddc& B) { return B.dII.p; }
  static const double* GG(const Bddc& B) { return B.dGG.p; }
  static const double* GC(const Bddc& B) { return B.dGC.p; }
};

// work vectors of one application z = M r (the preconditioner's own, or the
// allocation-free apply's static ones)
struct PrecBufs {
  double *tG, *vw, *gC, *uc, *work;
};

// One application z = M r: every per-subdomain stage is launched once per precision
// group -- all subdomains in one precision, or (mixed precision with some subdomains
// kept in FP64) the FP32 subdomains and then the FP64 ones; the coarse solve runs once
// between the Neumann and the prolongation stages.
template <int NC, int CL>
static void launch_preconditioner_cl(Bddc& B, const double* r, double* z, PcgScalars* sc, int with_dots,
                                     cudaStream_t s, const PrecBufs& bf) {
  const SubMeta sm = B.meta();
  const int ns = (int)B.mesh->n_sub;
  struct Group {
    bool f64;
    const int32_t* wl;
    int n;
  } gr[2];
  int ng = 0;
  if (!B.mixed)
    gr[ng++] = {true, nullptr, ns};
  else if (B.n_sub64 == 0)
    gr[ng++] = {false, nullptr, ns};
  else {
    gr[ng++] = {false, B.wl32.p, ns - B.n_sub64};
    gr[ng++] = {true, B.wl64.p, B.n_sub64};
  }
  size_t smem32 = 0, smem64 = 0;
  const SubLaunch L32 = sub_launch(B, 4, &smem32), L64 = sub_launch(B, 8, &smem64);
  // fn(TM tag, launch parameters, dynamic shared memory, subdomains) for each group
  auto each = [&](auto fn) {
    int off = 0;
    for (int k = 0; k < ng; ++k) {
      SubLaunch L = gr[k].f64 ? L64 : L32;
      L.wl = gr[k].wl;
      L.part_off = off;
      L.n_final = k == ng - 1 ? off + gr[k].n * CL : 0;
      if (gr[k].f64)
        fn(double(0), L, smem64, gr[k].n);
      else
        fn(float(0), L, smem32, gr[k].n);
      off += gr[k].n * CL;
    }
  };
  TimedLaunch t3, t4, t5, t6, t7;   // per-stage event timing (outside graph capture, when enabled)
  t3.begin("prec_interior", s);
  each([&](auto tag, const SubLaunch& L, size_t smem, int n) {
    using TM = decltype(tag);
    k_prec_interior1<TM, NC, CL><<<n * CL, kSubThreads, smem, s>>>(sm, LocalOps<TM>::II(B), r, bf.tG, sc, L);
    UFE_CHECK_LAUNCH();
  });
  t3.end(s);
  t4.begin("prec_neumann", s);
  each([&](auto tag, const SubLaunch& L, size_t smem, int n) {
    using TM = decltype(tag);
    k_prec_neumann<TM, NC, CL><<<n * CL, kSubThreads, smem, s>>>(sm, LocalOps<TM>::GG(B), LocalOps<TM>::GC(B), r,
                                                                 bf.tG, bf.vw, bf.gC, sc, L);
    UFE_CHECK_LAUNCH();
  });
  t4.end(s);
  if (B.n_coarse > 0) {
    t5.begin("coarse_solve", s);
    coarse_solve(B, bf.gC, bf.uc, bf.work, sc, s);
    t5.end(s);
    t6.begin("prec_prolong", s);
    each([&](auto tag, const SubLaunch& L, size_t smem, int n) {
      using TM = decltype(tag);
      k_prec_prolong<TM, NC, CL><<<n * CL, kSubThreads, smem, s>>>(sm, LocalOps<TM>::GC(B), bf.uc, bf.vw, sc, L);
      UFE_CHECK_LAUNCH();
    });
    t6.end(s);
  }
  t7.begin("prec_final", s);
  each([&](auto tag, const SubLaunch& L, size_t smem, int n) {
    using TM = decltype(tag);
    k_prec_final<TM, NC, CL><<<n * CL, kSubThreads, smem, s>>>(sm, LocalOps<TM>::II(B), r, bf.vw, z, B.part.p, sc,
                                                               L, with_dots);
    UFE_CHECK_LAUNCH();
  });
  t7.end(s);
}

// the cluster size the launch-shape tuner chose (Poisson; elasticity keeps four CTAs)
template <int NC>
static void launch_preconditioner(Bddc& B, const double* r, double* z, PcgScalars* sc, int with_dots, cudaStream_t s,
                                  const PrecBufs& bf) {
  if (NC == 1 && B.prec_cl == 2)
    launch_preconditioner_cl<NC, 2>(B, r, z, sc, with_dots, s, bf);
  else if (NC == 1 && B.prec_cl == 8)
    launch_preconditioner_cl<NC, 8>(B, r, z, sc, with_dots, s, bf);
  else
    launch_preconditioner_cl<NC, kCL>(B, r, z, sc, with_dots, s, bf);
}

// raise a kernel's dynamic shared-memory limit to what the device allows next to its
// static shared memory
template <typename K>
static void raise_smem_limit(K kernel, int optin) {
  cudaFuncAttributes fa;
  UFE_CUDA(cudaFuncGetAttributes(&fa, kernel));
  UFE_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes));
}

template <typename TM, int NC>
static void set_smem_limits_for(int optin) {
  raise_smem_limit(k_prec_interior1<TM, NC>, optin);
  raise_smem_limit(k_prec_neumann<TM, NC>, optin);
  raise_smem_limit(k_prec_final<TM, NC>, optin);
  raise_smem_limit(k_prec_prolong<TM, NC>, optin);
  if (NC == 1) {
    raise_smem_limit(k_prec_interior1<TM, NC, 2>, optin);
    raise_smem_limit(k_prec_neumann<TM, NC, 2>, optin);
    raise_smem_limit(k_prec_final<TM, NC, 2>, optin);
    raise_smem_limit(k_prec_prolong<TM, NC, 2>, optin);
    raise_smem_limit(k_prec_interior1<TM, NC, 8>, optin);
    raise_smem_limit(k_prec_neumann<TM, NC, 8>, optin);
    raise_smem_limit(k_prec_final<TM, NC, 8>, optin);
    raise_smem_limit(k_prec_prolong<TM, NC, 8>, optin);
  }
}

// The per-subdomain kernels take their dynamic shared memory from the problem; the
// opt-in limit is raised once per device to the largest a CTA may use (the limit
// does not change what a launch requests, so problems of different sizes can share
// it); each problem checks that its own request fits (with 16 KB left for the
// kernels' static shared memory).
void check_local_sizes(const Bddc& B) {
  size_t sd = 0, sf = 0;
  sub_launch(B, 8, &sd);
  sub_launch(B, 4, &sf);
  UFE_REQUIRE(std::max(sd, sf) <= (size_t)kMaxDynSmem, UFE_ERR_UNSUPPORTED,
              "local interface / interior sizes exceed one CTA's shared memory");
}

static void set_smem_limits(Bddc& B) {
  static std::mutex mu;
  static bool done[128] = {};
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
  check_local_sizes(B);
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  int optin = 0;
  UFE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  UFE_REQUIRE(optin >= kMaxDynSmem + 16 * 1024, UFE_ERR_UNSUPPORTED, "device offers too little shared memory per block");
  set_smem_limits_for<double, 1>(optin);
  set_smem_limits_for<float, 1>(optin);
  set_smem_limits_for<double, 3>(optin);
  set_smem_limits_for<float, 3>(optin);
  done[dev] = true;
}

// raise the flags the per-iteration kernels left behind (after the stream has synchronised)
static void check_device_status(Bddc& B) {
  int st = 0;
  UFE_CUDA(cudaMemcpyAsync(&st, B.status.p, sizeof(int), cudaMemcpyDeviceToHost, B.stream));
  UFE_CUDA(cudaStreamSynchronize(B.stream));
  if (st & DEV_TIMEOUT) throw Error{UFE_ERR_TIMEOUT, "a bulk copy of a local operator did not complete in time"};
}

static void precondition(Bddc& B, const double* r, double* z, PcgScalars* sc, int with_dots, cudaStream_t s) {
  const PrecBufs bf{B.tG.p, B.vw.p, B.gC.p, B.uc.p, B.cr.work.p};
  if (B.ncomp == 3)
    launch_preconditioner<3>(B, r, z, sc, with_dots, s, bf);
  else
    launch_preconditioner<1>(B, r, z, sc, with_dots, s, bf);
}

// ---------------------------------------------------------------------------
// Launch-shape tuner of the per-iteration preconditioner kernels (Poisson): CTAs per
// subdomain cluster (2, 4, 8) and row-stream stages per CTA (1, 2, 4).  The first
// set-up of a size class (device, precision, interior and interface sizes in steps of
// 32, subdomain count in powers of two) times each candidate with CUDA events (one
// warm-up, then three operator applies each followed by z = M r, as in an iteration,
// on the preconditioner's own work vectors, in five interleaved rounds, keeping each
// candidate's fastest) and caches the fastest for the process; later set-ups of the
// class reuse it.
// UFE_AUTOTUNE=0 keeps the default shape (4 CTAs, stages from the shared-memory budget),
// and so do problems of fewer than kTuneMinSubdomains subdomains: their stages are
// short, and a set of many small problems of different sizes (one solve each) would
// spend more time tuning its size classes than the shape can save.
// ---------------------------------------------------------------------------
constexpr int64_t kTuneMinSubdomains = 128;

static bool autotune_enabled() {
  const char* e = getenv("UFE_AUTOTUNE");
  return !(e && std::string(e) == "0");
}

static std::mutex g_tune_mu;
static std::map<std::array<int, 6>, std::pair<int, int>> g_tune_cache;   // size class -> (CTAs, stages)

static std::array<int, 6> tune_key(const Bddc& B) {
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  int nsb = 0;
  while ((1ll << nsb) < B.mesh->n_sub) ++nsb;
  return {dev, B.mixed ? 1 : 0, (B.max_nIv + 31) / 32, (B.max_nGv + 31) / 32, nsb, B.n_coarse > 0 ? 1 : 0};
}

// the launch shape where no timing is needed (fixed by the environment, untuned, or
// cached for the size class): sets it and returns true; false when it must be tuned
static bool known_shape(Bddc& B) {
  B.prec_cl = kCL;
  B.prec_stages = 0;
  if (B.ncomp != 1 || B.mesh->n_sub == 0) return true;
  if (const char* f = getenv("UFE_PREC_SHAPE")) {   // "cl,stages": a fixed shape (tests of every variant)
    int cl = kCL, st = 0;
    if (sscanf(f, "%d,%d", &cl, &st) == 2 && (cl == 2 || cl == 4 || cl == 8) && st >= 0 && st <= kMaxStages) {
      B.prec_cl = cl;
      B.prec_stages = st;
    }
    return true;
  }
  if (!autotune_enabled() || B.mesh->n_sub < kTuneMinSubdomains) return true;
  const std::array<int, 6> key = tune_key(B);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune_cache.find(key);
  if (it == g_tune_cache.end()) return false;
  B.prec_cl = it->second.first;
  B.prec_stages = it->second.second;
  return true;
}

void tune_preconditioner(Bddc& B) {
  if (known_shape(B)) return;
  const std::array<int, 6> key = tune_key(B);
  set_smem_limits(B);
  cudaStream_t s = B.stream;
  UFE_CUDA(cudaMemsetAsync(B.r.p, 0, (size_t)B.mesh->n_dof * 8, s));
  cudaEvent_t e0, e1;
  UFE_CUDA(cudaEventCreate(&e0));
  UFE_CUDA(cudaEventCreate(&e1));
  // every shape is timed in each of kRounds interleaved rounds (so that a slow moment of
  // the device does not single one out) and scored by its fastest round
  constexpr int kRounds = 5;
  const int shapes[9][2] = {{2, 1}, {2, 2}, {2, 4}, {4, 1}, {4, 2}, {4, 4}, {8, 1}, {8, 2}, {8, 4}};
  float score[9];
  for (float& v : score) v = 1e30f;
  std::pair<int, int> pick = {kCL, 0};
  const bool was_timing = timing_enabled();
  set_timing_enabled(false);   // the tuner's launches stay out of the instrumentation records
  try {
    for (int round = 0; round < kRounds; ++round)
      for (int k = 0; k < 9; ++k) {
        B.prec_cl = shapes[k][0];
        B.prec_stages = shapes[k][1];
        precondition(B, B.r.p, B.z.p, nullptr, 0, s);
        UFE_CUDA(cudaEventRecord(e0, s));
        // as in an iteration: the operator apply, then the preconditioner
        for (int rep = 0; rep < 3; ++rep) {
          system_apply(*B.sys, B.z.p, B.q.p, s);
          precondition(B, B.r.p, B.z.p, nullptr, 0, s);
        }
        UFE_CUDA(cudaEventRecord(e1, s));
        UFE_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        UFE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        score[k] = std::min(score[k], ms);
      }
    float best = 1e30f;
    for (int k = 0; k < 9; ++k)
      if (score[k] < best) {
        best = score[k];
        pick = {shapes[k][0], shapes[k][1]};
      }
  } catch (...) {
    set_timing_enabled(was_timing);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  set_timing_enabled(was_timing);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_device_status(B);
  B.prec_cl = pick.first;
  B.prec_stages = pick.second;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = pick;
}

void bddc_apply(Bddc& B, const double* r_dev, double* z_dev) {
  set_smem_limits(B);
  precondition(B, r_dev, z_dev, nullptr, 0, B.stream);
  check_device_status(B);
}

static void launch_iteration(Bddc& B, const OpArgs& a, cudaStream_t s) {
  const unsigned nb = (unsigned)a.n_tiles;
  const int64_t nv = (int64_t)B.ncomp * a.n_dof;
  if (B.ncomp == 3)
    k_dir_apply<3><<<nb, kTileThreads, 0, s>>>(a, B.z.p, B.p0.p, B.p1.p, B.q.p, B.part.p, B.sc.p);
  else
    k_dir_apply<1><<<nb, kTileThreads, 0, s>>>(a, B.z.p, B.p0.p, B.p1.p, B.q.p, B.part.p, B.sc.p);
  UFE_CHECK_LAUNCH();
  k_update<<<grid_for(nv, kApplyThreads), kApplyThreads, 0, s>>>(nv, B.x.p, B.r.p, B.p0.p, B.p1.p, B.q.p, B.part.p,
                                                                 B.sc.p);
  UFE_CHECK_LAUNCH();
  precondition(B, B.r.p, B.z.p, B.sc.p, 1, s);
}

static void launch_residual(Bddc& B, const OpArgs& a, int mode, double* r, double* out, cudaStream_t s) {
  const unsigned nb = (unsigned)a.n_tiles;
  if (B.ncomp == 3)
    k_residual<3><<<nb, kTileThreads, 0, s>>>(a, B.b.p, B.x.p, r, B.part.p, B.sc.p, mode, out);
  else
    k_residual<1><<<nb, kTileThreads, 0, s>>>(a, B.b.p, B.x.p, r, B.part.p, B.sc.p, mode, out);
  UFE_CHECK_LAUNCH();
}

// Records the whole solve of B into one graph (once per preconditioner): initial
// residual and preconditioner, a conditional while node around one iteration, the
// true residual.  The graph reads and writes only B's own buffers, so it is reused
// by every later solve.
static void build_solve_graph(Bddc& B) {
  if (B.solve_exec) return;
  const OpArgs a = op_args(*B.sys);
  // capture on library-owned streams (the caller's may be the legacy default stream,
  // which cannot be captured); the graph is launched on the caller's stream
  if (!B.cap_stream) UFE_CUDA(cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking));
  if (!B.cap_stream2) UFE_CUDA(cudaStreamCreateWithFlags(&B.cap_stream2, cudaStreamNonBlocking));
  cudaStream_t cs = B.cap_stream;
  long long captured = 0;
  bool body_open = false;
  UFE_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  g_capture_counter = &captured;
  try {
    launch_residual(B, a, 0, B.r.p, nullptr, cs);
    precondition(B, B.r.p, B.z.p, B.sc.p, 1, cs);
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    UFE_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphConditionalHandle h;
    UFE_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault));
    k_loop_cond<<<1, 1, 0, cs>>>(h, B.sc.p);
    UFE_CHECK_LAUNCH();
    B.k_init = captured;
    captured = 0;
    UFE_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    UFE_CUDA(cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &cp));
    UFE_CUDA(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    UFE_CUDA(cudaStreamBeginCaptureToGraph(B.cap_stream2, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    body_open = true;
    launch_iteration(B, a, B.cap_stream2);
    k_loop_cond<<<1, 1, 0, B.cap_stream2>>>(h, B.sc.p);
    UFE_CHECK_LAUNCH();
    cudaGraph_t body_out = nullptr;
    body_open = false;
    UFE_CUDA(cudaStreamEndCapture(B.cap_stream2, &body_out));
    B.k_body = captured;
    captured = 0;
    launch_residual(B, a, 1, nullptr, B.tres.p, cs);
    B.k_final = captured;
  } catch (...) {
    g_capture_counter = nullptr;
    cudaGraph_t junk = nullptr;
    if (body_open) cudaStreamEndCapture(B.cap_stream2, &junk);
    junk = nullptr;
    cudaStreamEndCapture(cs, &junk);
    if (junk) cudaGraphDestroy(junk);
    throw;
  }
  g_capture_counter = nullptr;
  cudaGraph_t gr = nullptr;
  UFE_CUDA(cudaStreamEndCapture(cs, &gr));
  const cudaError_t e = cudaGraphInstantiate(&B.solve_exec, gr, 0);
  cudaGraphDestroy(gr);
  UFE_CUDA(e);
}

bool solve_graph_early(Bddc& B) {
  if (B.solve_exec) return true;
  if (!known_shape(B)) return false;
  set_smem_limits(B);
  build_solve_graph(B);
  return true;
}

void solve_graph_reset(Bddc& B) {
  if (B.solve_exec) cudaGraphExecDestroy(B.solve_exec);
  B.solve_exec = nullptr;
}

// stage the inputs and launch the solve graph on stream s
static void solve_launch(Bddc& B, const double* b_dev, const double* x_dev, const ufe_solve_opts& o, cudaStream_t s) {
  const int64_t n = (int64_t)B.ncomp * B.mesh->n_dof;
  UFE_CUDA(cudaMemcpyAsync(B.b.p, b_dev, n * 8, cudaMemcpyDeviceToDevice, s));
  UFE_CUDA(cudaMemcpyAsync(B.x.p, x_dev, n * 8, cudaMemcpyDeviceToDevice, s));
  // initial scalars through the pinned mirror, so the copy does not synchronise the host
  PcgScalars init{};
  init.rtol = o.rtol;
  init.maxit = std::max(o.maxit, 0);
  init.flexible = o.flexible < 0 ? (B.mixed ? 1 : 0) : (o.flexible ? 1 : 0);
  *B.h_sc = init;
  UFE_CUDA(cudaMemcpyAsync(B.sc.p, B.h_sc, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
  UFE_CUDA(cudaGraphLaunch(B.solve_exec, s));
}

// read the state, copy x out (stream s must have the solve queued); returns the status
static ufe_status solve_finish(Bddc& B, double* x_dev, cudaStream_t s, ufe_solve_info* info, float ms) {
  const int64_t n = (int64_t)B.ncomp * B.mesh->n_dof;
  UFE_CUDA(cudaMemcpyAsync(B.h_sc, B.sc.p, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
  double tr[2] = {0.0, 0.0};
  UFE_CUDA(cudaMemcpyAsync(tr, B.tres.p, sizeof(tr), cudaMemcpyDeviceToHost, s));
  UFE_CUDA(cudaMemcpyAsync(x_dev, B.x.p, n * 8, cudaMemcpyDeviceToDevice, s));
  UFE_CUDA(cudaStreamSynchronize(s));
  const PcgScalars fin = *B.h_sc;
  if (fin.bb == 0.0) {
    UFE_CUDA(cudaMemsetAsync(x_dev, 0, n * 8, s));
    UFE_CUDA(cudaStreamSynchronize(s));
  }
  const long long body_runs = fin.passes > 0 ? (long long)fin.passes - 1 : 0;
  g_kernel_launches.fetch_add(B.k_init + body_runs * B.k_body + B.k_final, std::memory_order_relaxed);
  if (info) {
    info->iterations = fin.iter;
    info->converged = fin.done == 1;
    info->rel_residual = fin.bb > 0 ? std::sqrt(fin.rr / fin.bb) : 0.0;
    info->true_rel_residual = tr[1] > 0 ? std::sqrt(tr[0] / tr[1]) : 0.0;
    info->solve_ms = ms;
  }
  if (fin.done == 3) return UFE_ERR_BREAKDOWN;
  if (fin.done != 1) return UFE_ERR_NO_CONVERGENCE;
  return UFE_OK;
}

void pcg_solve(Bddc& B, const double* b_dev, double* x_dev, const ufe_solve_opts& o, ufe_solve_info* info) {
  cudaStream_t s = B.stream;
  set_smem_limits(B);
  build_solve_graph(B);
  cudaEvent_t e0, e1;
  UFE_CUDA(cudaEventCreate(&e0));
  UFE_CUDA(cudaEventCreate(&e1));
  UFE_CUDA(cudaEventRecord(e0, s));
  solve_launch(B, b_dev, x_dev, o, s);
  UFE_CUDA(cudaEventRecord(e1, s));
  UFE_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  UFE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const ufe_status st = solve_finish(B, x_dev, s, info, ms);
  check_device_status(B);
  if (st == UFE_ERR_BREAKDOWN) throw Error{UFE_ERR_BREAKDOWN, "PCG breakdown: p.Ap <= 0"};
  if (st == UFE_ERR_NO_CONVERGENCE) throw Error{UFE_ERR_NO_CONVERGENCE, "PCG did not reach the tolerance within maxit"};
}

// Many independent solves at once: every problem's solve graph is launched on one of
// a few library-owned streams, so the GPU runs the problems side by side; each
// stream first waits for its problems' own streams.  Returns the first non-OK status
// (all problems are solved and reported regardless).
constexpr int kBatchStreams = 16;
ufe_status pcg_solve_batched(int n, Bddc* const* Bs, const double* const* b_dev, double* const* x_dev,
                             const ufe_solve_opts& o, ufe_solve_info* infos) {
  static std::mutex mu;
  static cudaStream_t pool[128][kBatchStreams] = {};
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int k = 0; k < kBatchStreams; ++k)
      if (!pool[dev][k]) UFE_CUDA(cudaStreamCreateWithFlags(&pool[dev][k], cudaStreamNonBlocking));
  }
  for (int i = 0; i < n; ++i) {
    set_smem_limits(*Bs[i]);
    build_solve_graph(*Bs[i]);
  }
  std::vector<cudaEvent_t> ev(2 * (size_t)n, nullptr);
  struct Cleanup {
    std::vector<cudaEvent_t>& ev;
    ~Cleanup() {
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    }
  } cleanup{ev};
  for (int i = 0; i < n; ++i) {
    cudaStream_t si = pool[dev][i % kBatchStreams];
    cudaEvent_t ready;
    UFE_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    ev[2 * i] = ready;
    UFE_CUDA(cudaEventRecord(ready, Bs[i]->stream));
    UFE_CUDA(cudaStreamWaitEvent(si, ready, 0));
    solve_launch(*Bs[i], b_dev[i], x_dev[i], o, si);
    cudaEvent_t done;
    UFE_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    ev[2 * i + 1] = done;
    UFE_CUDA(cudaEventRecord(done, si));
  }
  // later work on each problem's stream follows its solve; added only after every
  // launch, since problems often share one stream and an earlier wait there would
  // chain the next problem's start to this one's end
  for (int i = 0; i < n; ++i) UFE_CUDA(cudaStreamWaitEvent(Bs[i]->stream, ev[2 * i + 1], 0));
  ufe_status first = UFE_OK;
  for (int i = 0; i < n; ++i) {
    const ufe_status st = solve_finish(*Bs[i], x_dev[i], pool[dev][i % kBatchStreams], infos ? infos + i : nullptr, 0.f);
    check_device_status(*Bs[i]);
    if (first == UFE_OK && st != UFE_OK) first = st;
  }
  return first;
}

// ---------------------------------------------------------------------------
// z = M r without any device allocation: the interface and coarse intermediates
// of the preconditioner live in one file-scope device array instead of the
// buffers ufe_bddc_setup allocates.  Limits: 262144 interface slots (sum over
// subdomains of their interface DOFs), 65536 subdomain coarse slots, 32768
// coarse DOFs -- 688128 doubles, about 5.5 MB held by every device that loads the
// library.  All calls share the array; calls that overlap on the GPU race.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocG = 262144, kNoAllocC = 65536, kNoAllocU = 32768;
// interface vectors, subdomain coarse parts, u_c and the coarse solver's work vector (2 n_c)
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocG + kNoAllocC + 3 * kNoAllocU];

// device address of the array for the current device, looked up once per device (the
// lookup may load this file's device code, which takes device memory: it is first made
// by ufe_bddc_setup through bddc_noalloc_prepare, never inside the allocation-free call)
static double* noalloc_scratch_ptr() {
  static std::mutex mu;
  static double* ptr[128] = {};
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    UFE_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    ptr[dev] = static_cast<double*>(p);
  }
  return ptr[dev];
}

void bddc_noalloc_prepare(Bddc& B) {
  set_smem_limits(B);
  noalloc_scratch_ptr();
  coarse_prepare();
}

void bddc_apply_noalloc(Bddc& B, const double* r_dev, double* z_dev) {
  const Mesh& m = *B.mesh;
  int dev = -1;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev == B.device, UFE_ERR_INVALID_ARG,
              "ufe_bddc_apply_noalloc: the current device (" + std::to_string(dev) +
                  ") is not the device the preconditioner was set up on (" + std::to_string(B.device) + ")");
  for (const void* ptr : {(const void*)r_dev, (const void*)z_dev}) {
    cudaPointerAttributes pa{};
    UFE_CUDA(cudaPointerGetAttributes(&pa, ptr));
    UFE_REQUIRE((pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) && pa.device == B.device,
                UFE_ERR_INVALID_ARG,
                "ufe_bddc_apply_noalloc: r and z must be device memory of the preconditioner's device");
  }
  UFE_REQUIRE(B.n_vGloc <= kNoAllocG, UFE_ERR_INVALID_ARG,
              "ufe_bddc_apply_noalloc: " + std::to_string(B.n_vGloc) + " interface slots exceed the static limit of " +
                  std::to_string(kNoAllocG));
  UFE_REQUIRE(B.n_Cloc <= kNoAllocC, UFE_ERR_INVALID_ARG,
              "ufe_bddc_apply_noalloc: " + std::to_string(B.n_Cloc) +
                  " subdomain coarse slots exceed the static limit of " + std::to_string(kNoAllocC));
  UFE_REQUIRE(B.n_coarse <= kNoAllocU, UFE_ERR_INVALID_ARG,
              "ufe_bddc_apply_noalloc: " + std::to_string(B.n_coarse) + " coarse DOFs exceed the static limit of " +
                  std::to_string(kNoAllocU));
  double* base = noalloc_scratch_ptr();
  double* tG = base;
  double* vw = base + kNoAllocG;
  double* gC = vw + kNoAllocG;
  double* uc = gC + kNoAllocC;
  set_smem_limits(B);
  // every entry of z is written by the kernels; clearing it first keeps the
  // behaviour identical to ufe_bddc_apply
  UFE_CUDA(cudaMemsetAsync(z_dev, 0, (size_t)B.ncomp * m.n_dof * sizeof(double), B.stream));
  // the same kernels in the same launch shape as ufe_bddc_apply, on the static vectors
  // (the cyclic-reduction coarse solver's work vector follows uc)
  const PrecBufs bf{tG, vw, gC, uc, uc + kNoAllocU};
  if (B.ncomp == 3)
    launch_preconditioner<3>(B, r_dev, z_dev, nullptr, 0, B.stream, bf);
  else
    launch_preconditioner<1>(B, r_dev, z_dev, nullptr, 0, B.stream, bf);
  check_device_status(B);
}

}  // namespace ufe
