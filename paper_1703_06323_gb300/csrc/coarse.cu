// Coarse problem of the BDDC preconditioner (Eq. bddc, second term): u_c = A_c^-1 r_c
// with A_c = sum_w R_cw^T A_c^w R_cw (Sect. 3.2), solved exactly in FP64, by one of:
//
// Dense: the explicit inverse (symmetric Gauss-Jordan), applied as one GEMV.  One
// launch per solve; the set-up costs n_c^3 / 2 FP64 FMAs, so it serves small coarse
// problems (the default up to 2048 coarse DOFs).
//
// Cyclic reduction:
// A_c couples two coarse DOFs only through a subdomain that both objects touch.  Give
// every coarse DOF the layer = the largest z block index among its subdomains: an
// object's subdomains all hold one of its nodes, so their z indices are a or {a-1, a},
// and two coupled DOFs therefore sit in the same or adjacent layers.  In layer order
// A_c is block tridiagonal:
//   D_p = A[p, p] (n_p x n_p),  F_p = A[p, p-1] (n_p x n_{p-1}),  A[p-1, p] = F_p^T.
// Block cyclic reduction eliminates the odd positions of the current list of layers
// in parallel, then recurses on the even ones.  Eliminating j with neighbours a < j < b:
//   X_j = D_j^-1                         (batched symmetric Gauss-Jordan)
//   T1_j = X_j F_j,  T2_j = X_j F_b^T,   W1_j = F_j^T X_j,  W2_j = F_b X_j
//   D_a -= W1_j F_j,  D_b -= W2_j F_b^T,  F'_b = -F_b T1_j   (new coupling b -> a)
// and the solve is one launch per level in each direction:
//   forward  (even q of the level):  r_q -= W2_{q-1} r_{q-1} + W1_{q+1} r_{q+1}
//   top:                             u_t  = X_t r_t
//   backward (odd j of the level):   u_j  = X_j r_j - T1_j u_{j-1} - T2_j u_{j+1}
// Every step is a dense FP64 matrix-vector product; all of them read ~5 blocks per
// eliminated layer instead of the n_c^2 entries of an explicit inverse, and the set-up
// factors n_c^3 / L^2-sized blocks instead of one n_c^3 matrix.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "bddc.cuh"
#include "dense.cuh"
#include "ufe_internal.cuh"

namespace ufe {

static __device__ __forceinline__ double cr_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
static void upload_vec(DBuf<T>& d, const std::vector<T>& v, cudaStream_t s) {
  d.alloc(std::max<size_t>(v.size(), 1), s);
  if (!v.empty()) UFE_CUDA(cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

// layer of every coarse DOF: the largest z block index of the subdomains in neigh(l)
__global__ void k_coarse_layer(int64_t n_coarse, GridGeom g, const int32_t* __restrict__ coarse_rep,
                               const uint8_t* __restrict__ coarse_nn, const int32_t* __restrict__ neigh,
                               const int32_t* __restrict__ sub_block, int32_t* __restrict__ layer) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_coarse) return;
  const int32_t rep = coarse_rep[l];
  int z = -1;
  for (int k = 0; k < coarse_nn[l]; ++k) z = max(z, sub_block[neigh[(int64_t)rep * 8 + k]] / (g.bx * g.by));
  layer[l] = z;
}

// sum of squares of the entries of A_c that couple layers more than one apart (zero by
// the argument above; checked once per set-up)
__global__ void k_coarse_band_check(int64_t n, int ld, const double* __restrict__ Ac, const int32_t* __restrict__ layer,
                                    double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (e < n * n) {
    const int64_t i = e / n, j = e % n;
    if (abs(layer[i] - layer[j]) > 1) {
      const double a = Ac[i * ld + j];
      v = a * a;
    }
  }
  v = cr_warp_sum(v);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

// dst (rows x cols, leading dimension ldd) = A_c[perm[r0 + i], perm[c0 + j]]
__global__ void k_coarse_gather_block(const double* __restrict__ Ac, int ldc, const int32_t* __restrict__ perm, int r0,
                                      int rows, int c0, int cols, double* __restrict__ dst, int ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e / cols), j = (int)(e % cols);
  dst[(int64_t)i * ldd + j] = Ac[(int64_t)perm[r0 + i] * ldc + perm[c0 + j]];
}

// dst = src^T for a list of blocks (one CTA row of 32 x 32 tiles per block)
struct TransDesc {
  int rows, cols;      // of src
  int lds, ldd;
  int64_t src, dst;
};
__global__ void k_coarse_transpose(const TransDesc* __restrict__ td, double* __restrict__ S) {
  const TransDesc d = td[blockIdx.y];
  const int tc = (d.cols + 31) / 32, tr = (d.rows + 31) / 32;
  if ((int)blockIdx.x >= tr * tc) return;
  const int r0 = (blockIdx.x / tc) * 32, c0 = (blockIdx.x % tc) * 32;
  __shared__ double t[32][33];
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int i = e / 32, j = e % 32;
    t[i][j] = (r0 + i < d.rows && c0 + j < d.cols) ? S[d.src + (int64_t)(r0 + i) * d.lds + c0 + j] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int i = e / 32, j = e % 32;   // dst row c0 + i, column r0 + j
    if (c0 + i < d.cols && r0 + j < d.rows) S[d.dst + (int64_t)(c0 + i) * d.ldd + r0 + j] = t[j][i];
  }
}

// r (CR order) gathered from the subdomain parts: r[p] = sum_k gC[cpos[l * 8 + k]], l = perm[p]
__global__ void k_coarse_gather(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ cpos,
                                const uint8_t* __restrict__ cnn, const double* __restrict__ gC, double* __restrict__ r,
                                const PcgScalars* sc) {
  if (sc && sc->done) return;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t l = perm[p];
  double s = 0.0;
  for (int k = 0; k < cnn[l]; ++k) s += gC[cpos[(int64_t)l * 8 + k]];
  r[p] = s;
}

// One step of the solve: every task writes rows [y, y + n) of the work vector V
// (r in V[0, n_c), u in V[n_c, 2 n_c)):
//   V[y + i] = (base >= 0 ? V[base + i] : 0) + sum_t sign_t sum_c M_t[i][c] V[x_t + c]
// and, for rows of u, also uc[perm[y - n_c + i]].  One warp per row; a launch's
// tasks read only rows that no task of the same launch writes.
__global__ void __launch_bounds__(256)
k_coarse_step(const CoarseTask* __restrict__ tasks, int ntask, const CoarseTerm* __restrict__ terms,
              const double* __restrict__ store, double* __restrict__ V, int64_t n_c, const int32_t* __restrict__ perm,
              double* __restrict__ uc, const PcgScalars* sc) {
  if (sc && sc->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int t = 0;
  while (t < ntask && row >= tasks[t].row0 + tasks[t].n) ++t;
  if (t >= ntask) return;
  const CoarseTask T = tasks[t];
  const int i = (int)(row - T.row0);
  double s = 0.0;
  for (int q = T.term0; q < T.term0 + T.nterm; ++q) {
    const CoarseTerm M = terms[q];
    const double* a = store + M.off + (int64_t)i * M.ld;
    const double* x = V + M.x;
    double acc = 0.0;
    for (int c = lane; c < M.cols; c += 32) acc = fma(a[c], x[c], acc);
    s += M.sign * acc;
  }
  s = cr_warp_sum(s);
  if (lane == 0) {
    const double v = (T.base >= 0 ? V[T.base + i] : 0.0) + s;
    V[T.y + i] = v;
    if (T.y >= n_c) uc[perm[T.y - n_c + i]] = v;
  }
}

// dense solver: r_c gathered from the subdomain parts into shared memory, then
// u_c = A_c^-1 r_c, one warp per row with eight independent 16-byte loads per lane
__global__ void k_coarse_dense(int64_t nco, int ldc, const double* __restrict__ Ainv, const int32_t* __restrict__ cpos,
                               const uint8_t* __restrict__ cnn, const double* __restrict__ gC, double* __restrict__ uc,
                               const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) char smem[];
  double* rc = reinterpret_cast<double*>(smem);
  // the (at most eight) subdomain parts of each coarse DOF are loaded together, two
  // coarse DOFs per thread and pass, and summed in subdomain order
  for (int64_t l0 = threadIdx.x; l0 < ldc; l0 += 2 * (int64_t)blockDim.x) {
    double v[2][8];
    int n[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t l = l0 + h * (int64_t)blockDim.x;
      n[h] = l < nco ? cnn[l] : 0;
      int4 pa = make_int4(0, 0, 0, 0), pb = pa;
      if (l < nco) {
        pa = *reinterpret_cast<const int4*>(cpos + l * 8);
        pb = *reinterpret_cast<const int4*>(cpos + l * 8 + 4);
      }
      const int p[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) v[h][k] = k < n[h] ? gC[p[k]] : 0.0;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t l = l0 + h * (int64_t)blockDim.x;
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < n[h]) s += v[h][k];
      if (l < ldc) rc[l] = s;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int U = 8;
  for (int64_t row = (int64_t)blockIdx.x * nw + wid; row < nco; row += (int64_t)gridDim.x * nw) {
    const double* Ar = Ainv + row * ldc;
    double s = 0.0;
    for (int c0 = lane * 2; c0 < ldc; c0 += 64 * U) {
      double2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + 64 * u;
        v[u] = c < ldc ? *reinterpret_cast<const double2*>(Ar + c) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + 64 * u;
        if (c < ldc) s += v[u].x * rc[c] + v[u].y * rc[c + 1];
      }
    }
    s = cr_warp_sum(s);
    if (lane == 0) uc[row] = s;
  }
}

void dense_coarse_gemv(int64_t n, int ld, const double* Ainv, const int32_t* cpos, const uint8_t* cnn,
                       const double* parts, double* u, const PcgScalars* sc, cudaStream_t s) {
  const size_t csm = (size_t)ld * 8;
  const unsigned cg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 1216));
  k_coarse_dense<<<cg, 256, csm, s>>>(n, ld, Ainv, cpos, cnn, parts, u, sc);
  UFE_CHECK_LAUNCH();
}

void coarse_solve(const Bddc& B, const double* gC, double* uc, double* work, const PcgScalars* sc, cudaStream_t s) {
  if (B.n_coarse == 0) return;
  if (B.ml.n2 > 0) {
    ml_coarse_solve(B, gC, uc, sc, s);
    return;
  }
  if (B.coarse_dense) {
    dense_coarse_gemv(B.n_coarse, B.ldc, B.Ac_inv.p, B.cpos.p, B.coarse_nn.p, gC, uc, sc, s);
    return;
  }
  const CoarseCR& C = B.cr;
  k_coarse_gather<<<grid_for(C.n, 256), 256, 0, s>>>(C.n, C.perm.p, B.cpos.p, B.coarse_nn.p, gC, work, sc);
  UFE_CHECK_LAUNCH();
  for (const CoarseStep& st : C.steps) {
    const unsigned blocks = (unsigned)((st.rows * 32 + 255) / 256);
    k_coarse_step<<<blocks, 256, 0, s>>>(C.tasks.p + st.task0, st.ntask, C.terms.p, C.store.p, work, C.n, C.perm.p, uc,
                                        sc);
    UFE_CHECK_LAUNCH();
  }
}

void coarse_prepare() {
  static std::mutex mu;
  static bool done[128] = {};
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaFuncAttributes fa;
  UFE_CUDA(cudaFuncGetAttributes(&fa, k_coarse_dense));
  UFE_CUDA(cudaFuncGetAttributes(&fa, k_coarse_gather));
  UFE_CUDA(cudaFuncGetAttributes(&fa, k_coarse_step));
  done[dev] = true;
}

namespace {

struct Layer {
  int n = 0;           // coarse DOFs
  int off = 0;         // first position in CR order
  int64_t D = -1;      // D_p / X_p block (n x ld)
  int64_t F = -1;      // coupling to the previous active layer (n x ld_prev)
  int ld = 0, ldF = 0;
};

}  // namespace

constexpr int64_t kDenseCoarseMax = 2048;

// first column with a nonzero in each row of the assembled coarse matrix (one warp per
// row; the diagonal is positive, so every row has one at or before its own column)
__global__ void k_first_nonzero(const double* __restrict__ A, int n, int ld, int32_t* __restrict__ first) {
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = A + (int64_t)row * ld;
  int f = row;
  for (int c0 = 0; c0 < row; c0 += 32) {
    const int c = c0 + lane;
    const unsigned m = __ballot_sync(0xffffffffu, c < row && a[c] != 0.0);
    if (m) {
      f = c0 + __ffs(m) - 1;
      break;
    }
  }
  if (lane == 0) first[row] = f;
}

void dense_coarse_prepare(int64_t n, int ld) {
  int dev = 0, optin = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  UFE_CUDA(cudaFuncGetAttributes(&fa, k_coarse_dense));
  const int64_t smem = 8 * (int64_t)ld;
  UFE_REQUIRE(smem <= optin - (int64_t)fa.sharedSizeBytes, UFE_ERR_UNSUPPORTED,
              "dense coarse solver: " + std::to_string(n) + " coarse DOFs exceed one CTA's shared memory");
  if (smem > 48 * 1024)   // the largest allowed, so that no later set-up lowers it under an earlier one
    UFE_CUDA(cudaFuncSetAttribute(k_coarse_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes));
}

static void dense_setup(Bddc& B, DBuf<double>& Ac, int ldc, cudaStream_t s) {
  const int64_t n = B.n_coarse;
  dense_coarse_prepare(n, ldc);
  // the status is read by coarse_check, so that the host is free while the inversion runs
  B.coarse_status.alloc(1, s);
  B.coarse_status.zero();
  // the coarse numbering follows the grid (objects in DOF order), so A_c is banded
  // and the inversion skips the blocks outside its envelope
  DBuf<int32_t> first;
  first.alloc(std::max<int64_t>(n, 1), s);
  k_first_nonzero<<<grid_for(n * 32, 256), 256, 0, s>>>(Ac.p, (int)n, ldc, first.p);
  UFE_CHECK_LAUNCH();
  std::vector<int32_t> first_h((size_t)n);
  UFE_CUDA(cudaMemcpyAsync(first_h.data(), first.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  UFE_CUDA(cudaStreamSynchronize(s));
  large_inverse<double>(Ac.p, (int)n, ldc, B.coarse_status.p, s, &first_h);
  B.Ac_inv.p = Ac.p;   // take the buffer over
  B.Ac_inv.n = Ac.n;
  B.Ac_inv.s = Ac.s;
  Ac.p = nullptr;
  Ac.n = 0;
  B.ldc = ldc;
  B.cr.bytes = 8.0 * (double)n * ldc;
  B.cr.inv_flops = std::pow((double)n, 3);
}

void coarse_check(Bddc& B) {
  if (!B.coarse_status.n) return;
  const int st = scalar_to_host(B.coarse_status.p, B.stream);
  B.coarse_status.release();
  UFE_REQUIRE(st == 0, UFE_ERR_SINGULAR_COARSE, "coarse matrix is not positive definite");
}

void coarse_setup(Bddc& B, DBuf<double>& Acb, int ldc, cudaStream_t s) {
  const Mesh& m = *B.mesh;
  CoarseCR& C = B.cr;
  const int64_t n = B.n_coarse;
  C.n = n;
  C.steps.clear();
  C.bytes = 0.0;
  C.inv_flops = 0.0;
  if (n == 0) return;
  B.coarse_dense = B.coarse_solver == UFE_COARSE_SOLVER_DENSE ||
                   (B.coarse_solver == UFE_COARSE_SOLVER_AUTO && n <= kDenseCoarseMax);
  if (B.coarse_dense) {
    dense_setup(B, Acb, ldc, s);
    return;
  }
  const double* Ac = Acb.p;
  // layers and the CR order
  DBuf<int32_t> dl;
  dl.alloc(n, s);
  k_coarse_layer<<<grid_for(n, 256), 256, 0, s>>>(n, m.g, B.coarse_rep.p, B.coarse_nn.p, m.neigh.p, m.sub_block.p,
                                                 dl.p);
  UFE_CHECK_LAUNCH();
  std::vector<int32_t> layer(n);
  {
    DBuf<double> bad;
    bad.alloc(1, s);
    bad.zero();
    k_coarse_band_check<<<grid_for(n * n, 256), 256, 0, s>>>(n, ldc, Ac, dl.p, bad.p);
    UFE_CHECK_LAUNCH();
    double hbad = 0.0;
    UFE_CUDA(cudaMemcpyAsync(layer.data(), dl.p, n * 4, cudaMemcpyDeviceToHost, s));
    UFE_CUDA(cudaMemcpyAsync(&hbad, bad.p, 8, cudaMemcpyDeviceToHost, s));
    UFE_CUDA(cudaStreamSynchronize(s));
    UFE_REQUIRE(hbad == 0.0, UFE_ERR_UNSUPPORTED, "coarse matrix couples non-adjacent layers");
  }
  std::vector<int32_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return layer[a] < layer[b]; });
  std::vector<Layer> L;
  for (int64_t p = 0; p < n;) {
    int64_t q = p;
    while (q < n && layer[perm[q]] == layer[perm[p]]) ++q;
    Layer ly;
    ly.n = (int)(q - p);
    ly.off = (int)p;
    ly.ld = pad4(ly.n);
    L.push_back(ly);
    p = q;
  }
  upload_vec(C.perm, perm, s);
  const int nl = (int)L.size();

  // storage plan: every block the set-up and the solve use, in one arena
  int64_t top = 0;
  auto take = [&](int rows, int ld) {
    const int64_t o = top;
    top += (int64_t)rows * ld;
    top = (top + 31) / 32 * 32;
    return o;
  };
  for (int p = 0; p < nl; ++p) {
    L[p].D = take(L[p].n, L[p].ld);
    if (p > 0) {
      L[p].ldF = L[p - 1].ld;
      L[p].F = take(L[p].n, L[p].ldF);
    }
  }
  // dry run of the reduction to size the per-level blocks
  struct Elim {
    int j, a, b;   // layer ids (a / b = -1 when absent)
    int64_t T1, T2, W1, W2, Fn;
  };
  std::vector<std::vector<Elim>> levels;
  std::vector<int> act(nl);
  for (int p = 0; p < nl; ++p) act[p] = p;
  {
    std::vector<int> cur = act;
    std::vector<int> ldF(nl), prev(nl, -1);
    for (int p = 1; p < nl; ++p) prev[p] = p - 1;
    while (cur.size() > 1) {
      std::vector<Elim> lev;
      for (size_t k = 1; k < cur.size(); k += 2) {
        Elim e{cur[k], cur[k - 1], k + 1 < cur.size() ? cur[k + 1] : -1, -1, -1, -1, -1, -1};
        const Layer &J = L[e.j], &A = L[e.a];
        e.T1 = take(J.n, A.ld);
        e.W1 = take(A.n, J.ld);
        if (e.b >= 0) {
          const Layer& Bl = L[e.b];
          e.T2 = take(J.n, Bl.ld);
          e.W2 = take(Bl.n, J.ld);
          e.Fn = take(Bl.n, A.ld);
        }
        lev.push_back(e);
      }
      levels.push_back(lev);
      std::vector<int> nxt;
      for (size_t k = 0; k < cur.size(); k += 2) nxt.push_back(cur[k]);
      cur.swap(nxt);
    }
  }
  C.store.alloc((size_t)std::max<int64_t>(top, 1), s);
  C.store.zero();
  double* S = C.store.p;
  for (int p = 0; p < nl; ++p) {
    const Layer& ly = L[p];
    k_coarse_gather_block<<<grid_for((int64_t)ly.n * ly.n, 256), 256, 0, s>>>(Ac, ldc, C.perm.p, ly.off, ly.n, ly.off,
                                                                             ly.n, S + ly.D, ly.ld);
    UFE_CHECK_LAUNCH();
    if (p > 0) {
      const Layer& pv = L[p - 1];
      k_coarse_gather_block<<<grid_for((int64_t)ly.n * pv.n, 256), 256, 0, s>>>(Ac, ldc, C.perm.p, ly.off, ly.n,
                                                                               pv.off, pv.n, S + ly.F, ly.ldF);
      UFE_CHECK_LAUNCH();
    }
  }

  // every layer is inverted once: one status slot per layer, read after the last inversion
  DBuf<int> st;
  st.alloc(std::max(nl, 1), s);
  st.zero();
  int n_inv = 0;
  auto invert = [&](const std::vector<int>& ids) {
    std::vector<InvDesc> d;
    for (int id : ids) {
      d.push_back({L[id].n, L[id].ld, L[id].D});
      C.inv_flops += std::pow((double)L[id].n, 3);
    }
    batched_inverse<double>(d, S, st.p + n_inv, s);
    n_inv += (int)ids.size();
  };
  // coupling of layer b to its current left neighbour: F[b] (storage may move to Fn)
  std::vector<int64_t> Fcur(nl, -1);
  std::vector<int> Fld(nl, 0);
  for (int p = 1; p < nl; ++p) {
    Fcur[p] = L[p].F;
    Fld[p] = L[p].ldF;
  }
  for (auto& lev : levels) {
    std::vector<int> ids;
    for (auto& e : lev) ids.push_back(e.j);
    invert(ids);
    std::vector<GemmDesc> t1, t2, da, dbf;
    std::vector<TransDesc> tw;
    for (auto& e : lev) {
      const Layer &J = L[e.j], &A = L[e.a];
      // T1 = X_j F_j (n_j x n_a);  W1 = T1^T (X_j symmetric);  D_a -= F_j^T T1
      t1.push_back({J.n, A.n, J.n, J.ld, Fld[e.j], A.ld, J.D, Fcur[e.j], e.T1});
      tw.push_back({J.n, A.n, A.ld, J.ld, e.T1, e.W1});
      da.push_back({A.n, A.n, J.n, Fld[e.j], A.ld, A.ld, Fcur[e.j], e.T1, A.D});
      if (e.b >= 0) {
        const Layer& Bl = L[e.b];
        // T2 = X_j F_b^T (n_j x n_b);  W2 = T2^T;  D_b -= F_b T2;  F'_b = -F_b T1 (into zeros)
        t2.push_back({J.n, Bl.n, J.n, J.ld, Fld[e.b], Bl.ld, J.D, Fcur[e.b], e.T2});
        tw.push_back({J.n, Bl.n, Bl.ld, J.ld, e.T2, e.W2});
        dbf.push_back({Bl.n, Bl.n, J.n, Fld[e.b], Bl.ld, Bl.ld, Fcur[e.b], e.T2, Bl.D});
        dbf.push_back({Bl.n, A.n, J.n, Fld[e.b], A.ld, A.ld, Fcur[e.b], e.T1, e.Fn});
      }
    }
    batched_gemm<double>(false, false, t1, S, S, S, 1.0, 0.0, s);
    if (!t2.empty()) batched_gemm<double>(false, true, t2, S, S, S, 1.0, 0.0, s);
    {
      DBuf<TransDesc> dtw;
      upload_vec(dtw, tw, s);
      int mt = 0;
      for (const TransDesc& d : tw) mt = std::max(mt, ((d.rows + 31) / 32) * ((d.cols + 31) / 32));
      k_coarse_transpose<<<dim3(mt, (unsigned)tw.size()), 256, 0, s>>>(dtw.p, S);
      UFE_CHECK_LAUNCH();
    }
    batched_gemm<double>(true, false, da, S, S, S, -1.0, 1.0, s);
    if (!dbf.empty()) batched_gemm<double>(false, false, dbf, S, S, S, -1.0, 1.0, s);
    for (auto& e : lev)
      if (e.b >= 0) {
        Fcur[e.b] = e.Fn;
        Fld[e.b] = L[e.a].ld;
      }
  }
  // the last active layer
  int topl = 0;
  {
    std::vector<int> cur = act;
    while (cur.size() > 1) {
      std::vector<int> nxt;
      for (size_t k = 0; k < cur.size(); k += 2) nxt.push_back(cur[k]);
      cur.swap(nxt);
    }
    topl = cur[0];
    invert({topl});
    std::vector<int> hs(n_inv);
    UFE_CUDA(cudaMemcpyAsync(hs.data(), st.p, n_inv * 4, cudaMemcpyDeviceToHost, s));
    UFE_CUDA(cudaStreamSynchronize(s));
    for (int v : hs) UFE_REQUIRE(v == 0, UFE_ERR_SINGULAR_COARSE, "coarse matrix is not positive definite");
  }

  // the solve: forward levels, top, backward levels (reverse)
  std::vector<CoarseTask> tasks;
  std::vector<CoarseTerm> terms;
  const int64_t U0 = n;   // u rows start here in the work vector
  auto add_step = [&](const std::vector<CoarseTask>& tk) {
    CoarseStep cs;
    cs.task0 = (int)tasks.size();
    cs.ntask = (int)tk.size();
    int64_t rows = 0;
    for (CoarseTask t : tk) {
      t.row0 = rows;
      rows += t.n;
      tasks.push_back(t);
    }
    cs.rows = rows;
    C.steps.push_back(cs);
  };
  auto term = [&](int64_t off, int ld, int cols, int64_t x, double sign) { terms.push_back({off, ld, cols, x, sign}); };
  double bytes = 0.0;
  for (auto& lev : levels) {
    // even q neighbours of this level: r_q -= W2_{q-1} r_{q-1} + W1_{q+1} r_{q+1}
    std::vector<int> evens;
    for (auto& e : lev) {
      evens.push_back(e.a);
      if (e.b >= 0) evens.push_back(e.b);
    }
    std::sort(evens.begin(), evens.end());
    evens.erase(std::unique(evens.begin(), evens.end()), evens.end());
    std::vector<CoarseTask> tk;
    for (int q : evens) {
      CoarseTask t{};
      t.y = L[q].off;
      t.base = L[q].off;
      t.n = L[q].n;
      t.term0 = (int)terms.size();
      for (auto& e : lev) {
        if (e.b == q) {   // left neighbour j of q
          term(e.W2, L[e.j].ld, L[e.j].n, L[e.j].off, -1.0);
          bytes += 8.0 * L[q].n * L[e.j].n;
        }
        if (e.a == q) {   // right neighbour j of q
          term(e.W1, L[e.j].ld, L[e.j].n, L[e.j].off, -1.0);
          bytes += 8.0 * L[q].n * L[e.j].n;
        }
      }
      t.nterm = (int)terms.size() - t.term0;
      tk.push_back(t);
    }
    add_step(tk);
  }
  {
    CoarseTask t{};
    t.y = U0 + L[topl].off;
    t.base = -1;
    t.n = L[topl].n;
    t.term0 = (int)terms.size();
    term(L[topl].D, L[topl].ld, L[topl].n, L[topl].off, 1.0);
    bytes += 8.0 * L[topl].n * L[topl].n;
    t.nterm = 1;
    add_step({t});
  }
  for (auto it = levels.rbegin(); it != levels.rend(); ++it) {
    std::vector<CoarseTask> tk;
    for (auto& e : *it) {
      const Layer& J = L[e.j];
      CoarseTask t{};
      t.y = U0 + J.off;
      t.base = -1;
      t.n = J.n;
      t.term0 = (int)terms.size();
      term(J.D, J.ld, J.n, J.off, 1.0);
      term(e.T1, L[e.a].ld, L[e.a].n, U0 + L[e.a].off, -1.0);
      bytes += 8.0 * J.n * (J.n + L[e.a].n);
      if (e.b >= 0) {
        term(e.T2, L[e.b].ld, L[e.b].n, U0 + L[e.b].off, -1.0);
        bytes += 8.0 * J.n * L[e.b].n;
      }
      t.nterm = (int)terms.size() - t.term0;
      tk.push_back(t);
    }
    add_step(tk);
  }
  upload_vec(C.tasks, tasks, s);
  upload_vec(C.terms, terms, s);
  C.bytes = bytes;
  C.nlayers = nl;
  C.nlevels = (int)levels.size();
  C.work.alloc(2 * n, s);
}

}  // namespace ufe
