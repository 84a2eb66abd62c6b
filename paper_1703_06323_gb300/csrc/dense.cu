// Batched dense linear algebra for the local BDDC operators.
//
// batched_gemm: one CTA per 64x64 output tile of one problem; 16-deep k slabs
// staged in shared memory; each of the 256 threads owns a 4x4 register tile.
//
// Inversion: blocked Gauss-Jordan in place.  For each diagonal block K (width 32):
//   A_KK <- A_KK^-1,  A_Kj <- A_KK^-1 A_Kj,  A_ij <- A_ij - A_iK A_Kj,  A_iK <- -A_iK A_KK^-1
// (i, j outside K).  After the last block A holds A^-1.  Without pivoting this is
// stable for SPD matrices, whose pivots are Schur complements and stay positive;
// a pivot <= 0 (or not finite) flags the matrix as singular.
#include <vector>

#include "dense.cuh"

namespace ufe {

constexpr int kTile = 64, kSlab = 16, kGemmThreads = 256, kNB = 32;

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads)
k_batched_gemm(const GemmDesc* __restrict__ descs, const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C,
               T alpha, T beta) {
  const GemmDesc d = descs[blockIdx.y];
  const int tiles_n = (d.n + kTile - 1) / kTile;
  const int tiles_m = (d.m + kTile - 1) / kTile;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int i0 = (blockIdx.x / tiles_n) * kTile, j0 = (blockIdx.x % tiles_n) * kTile;
  __shared__ T As[kSlab][kTile + 1];
  __shared__ T Bs[kSlab][kTile + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  const T* Ab = A + d.a;
  const T* Bb = B + d.b;
  for (int l0 = 0; l0 < d.k; l0 += kSlab) {
    for (int e = threadIdx.x; e < kSlab * kTile; e += kGemmThreads) {
      const int l = e / kTile, r = e % kTile;
      const int gi = i0 + r, gl = l0 + l;
      T av = T(0);
      if (gi < d.m && gl < d.k) av = TA ? Ab[(int64_t)gl * d.lda + gi] : Ab[(int64_t)gi * d.lda + gl];
      As[l][r] = av;
      const int gj = j0 + r;
      T bv = T(0);
      if (gj < d.n && gl < d.k) bv = TB ? Bb[(int64_t)gj * d.ldb + gl] : Bb[(int64_t)gl * d.ldb + gj];
      Bs[l][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < kSlab; ++l) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[l][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[l][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
  T* Cb = C + d.c;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= d.m) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj >= d.n) continue;
      T* cp = Cb + (int64_t)gi * d.ldc + gj;
      *cp = alpha * acc[a][b] + (beta == T(0) ? T(0) : beta * *cp);
    }
  }
}

template <typename T>
void batched_gemm(bool transA, bool transB, const std::vector<GemmDesc>& descs, const T* A, const T* B, T* C,
                  T alpha, T beta, cudaStream_t s) {
  if (descs.empty()) return;
  int max_tiles = 0;
  for (const auto& d : descs) {
    const int t = ((d.m + kTile - 1) / kTile) * ((d.n + kTile - 1) / kTile);
    if (t > max_tiles) max_tiles = t;
  }
  if (max_tiles == 0) return;
  DBuf<GemmDesc> dd;
  dd.alloc(descs.size(), s);
  UFE_CUDA(cudaMemcpyAsync(dd.p, descs.data(), descs.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, s));
  dim3 grid(max_tiles, (unsigned)descs.size());
  if (!transA && !transB) {
    k_batched_gemm<T, false, false><<<grid, kGemmThreads, 0, s>>>(dd.p, A, B, C, alpha, beta);
    UFE_CHECK_LAUNCH();
  }
  else if (transA && !transB) {
    k_batched_gemm<T, true, false><<<grid, kGemmThreads, 0, s>>>(dd.p, A, B, C, alpha, beta);
    UFE_CHECK_LAUNCH();
  }
  else if (!transA && transB) {
    k_batched_gemm<T, false, true><<<grid, kGemmThreads, 0, s>>>(dd.p, A, B, C, alpha, beta);
    UFE_CHECK_LAUNCH();
  }
  else {
    k_batched_gemm<T, true, true><<<grid, kGemmThreads, 0, s>>>(dd.p, A, B, C, alpha, beta);
    UFE_CHECK_LAUNCH();
  }
  // the descriptor buffer is released stream-ordered after the kernel
}

// ---------------------------------------------------------------------------
// Gauss-Jordan building blocks (CTA-level); all take the block column k0, kb
// ---------------------------------------------------------------------------

// invert the kb x kb diagonal block into Dinv (shared memory); returns false if singular
template <typename T>
__device__ bool gj_diag(T* A, int ld, int k0, int kb, T (*D)[kNB + 1]) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    D[r][c] = A[(int64_t)(k0 + r) * ld + k0 + c];
  }
  __syncthreads();
  for (int p = 0; p < kb; ++p) {
    const T piv = D[p][p];
    if (!(piv > T(0)) || !isfinite((double)piv)) {
      if (threadIdx.x == 0) bad = 1;
    }
    const T inv = T(1) / piv;
    __syncthreads();
    // row p
    for (int c = threadIdx.x; c < kb; c += blockDim.x)
      if (c != p) D[p][c] *= inv;
    __syncthreads();
    // other rows
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int r = e / kb, c = e % kb;
      if (r == p || c == p) continue;
      D[r][c] -= D[r][p] * D[p][c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < kb; r += blockDim.x)
      if (r != p) D[r][p] = -D[r][p] * inv;
    if (threadIdx.x == 0) D[p][p] = inv;
    __syncthreads();
  }
  const bool ok = bad == 0;
  __syncthreads();
  return ok;
}

// A_Kj <- Dinv A_Kj for the columns j in [jb, je) outside K
template <typename T>
__device__ void gj_row_panel(T* A, int ld, int n, int k0, int kb, const T (*D)[kNB + 1], int jb, int je, int tid,
                             int nthreads) {
  for (int j = jb + tid; j < je; j += nthreads) {
    if (j >= k0 && j < k0 + kb) continue;
    T col[kNB];
#pragma unroll
    for (int r = 0; r < kNB; ++r) col[r] = r < kb ? A[(int64_t)(k0 + r) * ld + j] : T(0);
#pragma unroll 4
    for (int r = 0; r < kb; ++r) {
      T sacc = T(0);
#pragma unroll
      for (int c = 0; c < kNB; ++c) sacc += D[r][c < kb ? c : 0] * (c < kb ? col[c] : T(0));
      A[(int64_t)(k0 + r) * ld + j] = sacc;
    }
  }
  (void)n;
}

// A_iK <- -A_iK Dinv for the rows i in [ib, ie) outside K
template <typename T>
__device__ void gj_col_panel(T* A, int ld, int k0, int kb, const T (*D)[kNB + 1], int ib, int ie, int tid,
                             int nthreads) {
  for (int i = ib + tid; i < ie; i += nthreads) {
    if (i >= k0 && i < k0 + kb) continue;
    T row[kNB];
#pragma unroll
    for (int c = 0; c < kNB; ++c) row[c] = c < kb ? A[(int64_t)i * ld + k0 + c] : T(0);
#pragma unroll 4
    for (int c = 0; c < kb; ++c) {
      T sacc = T(0);
#pragma unroll
      for (int r = 0; r < kNB; ++r) sacc += (r < kb ? row[r] : T(0)) * D[r < kb ? r : 0][c];
      A[(int64_t)i * ld + k0 + c] = -sacc;
    }
  }
}

// A_ij -= A_iK A_Kj on one 64x64 tile (i0, j0), skipping i or j inside K
template <typename T>
__device__ void gj_update_tile(T* A, int ld, int n, int k0, int kb, int i0, int j0, T (*As)[kTile + 1],
                               T (*Bs)[kTile + 1]) {
  for (int e = threadIdx.x; e < kNB * kTile; e += blockDim.x) {
    const int l = e / kTile, r = e % kTile;
    const int gi = i0 + r, gj = j0 + r;
    As[l][r] = (l < kb && gi < n) ? A[(int64_t)gi * ld + k0 + l] : T(0);
    Bs[l][r] = (l < kb && gj < n) ? A[(int64_t)(k0 + l) * ld + gj] : T(0);
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int l = 0; l < kb; ++l) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[l][ty + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[l][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= n || (gi >= k0 && gi < k0 + kb)) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj >= n || (gj >= k0 && gj < k0 + kb)) continue;
      A[(int64_t)gi * ld + gj] -= acc[a][b];
    }
  }
  __syncthreads();
}

// one CTA inverts one matrix of the batch
template <typename T>
__global__ void __launch_bounds__(kGemmThreads) k_batched_inverse(const InvDesc* __restrict__ descs, T* base, int* status) {
  const InvDesc d = descs[blockIdx.x];
  if (d.n <= 0) return;
  T* A = base + d.off;
  __shared__ T D[kNB][kNB + 1];
  __shared__ T As[kNB][kTile + 1];
  __shared__ T Bs[kNB][kTile + 1];
  bool ok = true;
  for (int k0 = 0; k0 < d.n; k0 += kNB) {
    const int kb = min(kNB, d.n - k0);
    ok = gj_diag<T>(A, d.ld, k0, kb, D) && ok;
    gj_row_panel<T>(A, d.ld, d.n, k0, kb, D, 0, d.n, threadIdx.x, blockDim.x);
    __syncthreads();
    const int tiles = (d.n + kTile - 1) / kTile;
    for (int t = 0; t < tiles * tiles; ++t) gj_update_tile<T>(A, d.ld, d.n, k0, kb, (t / tiles) * kTile, (t % tiles) * kTile, As, Bs);
    gj_col_panel<T>(A, d.ld, k0, kb, D, 0, d.n, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int r = e / kb, c = e % kb;
      A[(int64_t)(k0 + r) * d.ld + k0 + c] = D[r][c];
    }
    __syncthreads();
  }
  if (!ok && threadIdx.x == 0) atomicOr(status + blockIdx.x, DEV_SINGULAR);
}

template <typename T>
void batched_inverse(const std::vector<InvDesc>& descs, T* base, int* status, cudaStream_t s) {
  if (descs.empty()) return;
  DBuf<InvDesc> dd;
  dd.alloc(descs.size(), s);
  UFE_CUDA(cudaMemcpyAsync(dd.p, descs.data(), descs.size() * sizeof(InvDesc), cudaMemcpyHostToDevice, s));
  k_batched_inverse<T><<<(unsigned)descs.size(), kGemmThreads, 0, s>>>(dd.p, base, status);
  UFE_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// one large matrix: the same four steps, each spread over the grid
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_large_diag(T* A, int ld, int k0, int kb, T* Dout, int* status) {
  __shared__ T D[kNB][kNB + 1];
  const bool ok = gj_diag<T>(A, ld, k0, kb, D);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) Dout[e] = D[e / kNB][e % kNB];
  if (!ok && threadIdx.x == 0) atomicOr(status, DEV_SINGULAR);
}

template <typename T>
__device__ void load_D(const T* Dg, T (*D)[kNB + 1]) {
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) D[e / kNB][e % kNB] = Dg[e];
  __syncthreads();
}

template <typename T>
__global__ void k_large_row_panel(T* A, int ld, int n, int k0, int kb, const T* Dg) {
  __shared__ T D[kNB][kNB + 1];
  load_D<T>(Dg, D);
  gj_row_panel<T>(A, ld, n, k0, kb, D, 0, n, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kGemmThreads) k_large_update(T* A, int ld, int n, int k0, int kb) {
  __shared__ T As[kNB][kTile + 1];
  __shared__ T Bs[kNB][kTile + 1];
  const int tiles = (n + kTile - 1) / kTile;
  for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x)
    gj_update_tile<T>(A, ld, n, k0, kb, (t / tiles) * kTile, (t % tiles) * kTile, As, Bs);
}

template <typename T>
__global__ void k_large_col_panel(T* A, int ld, int n, int k0, int kb, const T* Dg) {
  __shared__ T D[kNB][kNB + 1];
  load_D<T>(Dg, D);
  gj_col_panel<T>(A, ld, k0, kb, D, 0, n, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  if (blockIdx.x == 0)
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x)
      A[(int64_t)(k0 + e / kb) * ld + k0 + e % kb] = D[e / kb][e % kb];
}

template <typename T>
void large_inverse(T* A, int n, int ld, int* status, cudaStream_t s) {
  if (n <= 0) return;
  DBuf<T> Dg;
  Dg.alloc(kNB * kNB, s);
  const int tiles = (n + kTile - 1) / kTile;
  const unsigned upd_grid = (unsigned)std::min(tiles * tiles, 152 * 8);
  const unsigned panel_grid = (unsigned)std::max(1, std::min((n + 255) / 256, 152 * 4));
  for (int k0 = 0; k0 < n; k0 += kNB) {
    const int kb = std::min(kNB, n - k0);
    k_large_diag<T><<<1, 256, 0, s>>>(A, ld, k0, kb, Dg.p, status);
    UFE_CHECK_LAUNCH();
    k_large_row_panel<T><<<panel_grid, 256, 0, s>>>(A, ld, n, k0, kb, Dg.p);
    UFE_CHECK_LAUNCH();
    k_large_update<T><<<upd_grid, kGemmThreads, 0, s>>>(A, ld, n, k0, kb);
    UFE_CHECK_LAUNCH();
    k_large_col_panel<T><<<panel_grid, 256, 0, s>>>(A, ld, n, k0, kb, Dg.p);
    UFE_CHECK_LAUNCH();
  }
}

template void batched_gemm<double>(bool, bool, const std::vector<GemmDesc>&, const double*, const double*, double*,
                                   double, double, cudaStream_t);
template void batched_gemm<float>(bool, bool, const std::vector<GemmDesc>&, const float*, const float*, float*, float,
                                  float, cudaStream_t);
template void batched_inverse<double>(const std::vector<InvDesc>&, double*, int*, cudaStream_t);
template void batched_inverse<float>(const std::vector<InvDesc>&, float*, int*, cudaStream_t);
template void large_inverse<double>(double*, int, int, int*, cudaStream_t);

}  // namespace ufe
