// Batched dense linear algebra for the local BDDC operators.
//
// batched_gemm: one CTA per 64x64 output tile of one problem; 16-deep k slabs
// staged in shared memory; each of the 256 threads owns a 4x4 register tile.
//
// Inversion: blocked Gauss-Jordan.  For each diagonal block K (width 64):
//   A_KK <- A_KK^-1,  A_Kj <- A_KK^-1 A_Kj,  A_ij <- A_ij - A_iK A_KK^-1 A_Kj,  A_iK <- -A_iK A_KK^-1
// (i, j outside K).  After the last block A holds A^-1.  Without pivoting this is
// stable for SPD matrices, whose pivots are Schur complements and stay positive;
// a pivot <= 0 (or not finite) flags the matrix as singular.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "dense.cuh"

namespace ufe {

constexpr int kTile = 64, kSlab = 16, kGemmThreads = 256;

// C tile of TS x TS per CTA (TS = 64: 4 x 4 outputs per thread; TS = 16: one output
// per thread, for batches too small to fill the GPU with 64 x 64 tiles)
template <typename T, bool TA, bool TB, int TS>
__global__ void __launch_bounds__(kGemmThreads)
k_batched_gemm(const GemmDesc* __restrict__ descs, const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C,
               T alpha, T beta) {
  constexpr int RB = TS / 16;
  const GemmDesc d = descs[blockIdx.y];
  const int tiles_n = (d.n + TS - 1) / TS;
  const int tiles_m = (d.m + TS - 1) / TS;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int i0 = (blockIdx.x / tiles_n) * TS, j0 = (blockIdx.x % tiles_n) * TS;
  __shared__ T As[kSlab][TS + 1];
  __shared__ T Bs[kSlab][TS + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[RB][RB];
#pragma unroll
  for (int a = 0; a < RB; ++a)
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[a][b] = T(0);
  const T* Ab = A + d.a;
  const T* Bb = B + d.b;
  for (int l0 = 0; l0 < d.k; l0 += kSlab) {
    for (int e = threadIdx.x; e < kSlab * TS; e += kGemmThreads) {
      const int l = e / TS, r = e % TS;
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
      T av[RB], bv[RB];
#pragma unroll
      for (int a = 0; a < RB; ++a) av[a] = As[l][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < RB; ++b) bv[b] = Bs[l][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
  T* Cb = C + d.c;
#pragma unroll
  for (int a = 0; a < RB; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= d.m) continue;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj >= d.n) continue;
      T* cp = Cb + (int64_t)gi * d.ldc + gj;
      *cp = alpha * acc[a][b] + (beta == T(0) ? T(0) : beta * *cp);
    }
  }
}

// streaming multiprocessors of the current device (looked up once per device)
static int sm_count() {
  static std::mutex mu;
  static int n[128] = {};
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
  std::lock_guard<std::mutex> lock(mu);
  if (!n[dev]) UFE_CUDA(cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev));
  return n[dev];
}

template <typename T>
void batched_gemm(bool transA, bool transB, const std::vector<GemmDesc>& descs, const T* A, const T* B, T* C,
                  T alpha, T beta, cudaStream_t s) {
  if (descs.empty()) return;
  auto tiles = [&](int ts, int64_t* total) {
    int mx = 0;
    *total = 0;
    for (const auto& d : descs) {
      const int t = ((d.m + ts - 1) / ts) * ((d.n + ts - 1) / ts);
      mx = std::max(mx, t);
      *total += t;
    }
    return mx;
  };
  int64_t total64 = 0, total16 = 0;
  const int max64 = tiles(kTile, &total64);
  if (max64 == 0) return;
  // batches that give fewer 64 x 64 tiles than two per SM (the coarse layers) take
  // 16 x 16 tiles: FP64 runs a few FMA per clock per SM, so work must spread out
  const bool small = total64 < 2 * (int64_t)sm_count();
  const int max16 = tiles(16, &total16);
  DBuf<GemmDesc> dd;
  dd.alloc(descs.size(), s);
  UFE_CUDA(cudaMemcpyAsync(dd.p, descs.data(), descs.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, s));
  const dim3 grid(small ? max16 : max64, (unsigned)descs.size());
  auto go = [&](auto kernel) {
    kernel<<<grid, kGemmThreads, 0, s>>>(dd.p, A, B, C, alpha, beta);
    UFE_CHECK_LAUNCH();
  };
  if (!transA && !transB)
    small ? go(k_batched_gemm<T, false, false, 16>) : go(k_batched_gemm<T, false, false, kTile>);
  else if (transA && !transB)
    small ? go(k_batched_gemm<T, true, false, 16>) : go(k_batched_gemm<T, true, false, kTile>);
  else if (!transA && transB)
    small ? go(k_batched_gemm<T, false, true, 16>) : go(k_batched_gemm<T, false, true, kTile>);
  else
    small ? go(k_batched_gemm<T, true, true, 16>) : go(k_batched_gemm<T, true, true, kTile>);
  // the descriptor buffer is released stream-ordered after the kernel
}

// ---------------------------------------------------------------------------
// Batched blocked Gauss-Jordan inversion, one block column (width NB) per step,
// three launches per step over the whole batch:
//   panel:     the old row panel R_K* = A_K* and Q_K* = D^-1 A_K*;
//   update:    every tile (I <= J) of the next iterate, A_IJ - P_IK Q_KJ, Q_KJ,
//              -P_IK D^-1 or D^-1, with P_IK = +-R_KI^T, and its mirror tile, except
//              block row / column K+1;
//   lookahead: block row / column K+1 of the same update, with the diagonal tile
//              (K+1, K+1) kept in shared memory and inverted there (D^-1 of the next
//              step; register-blocked Gauss-Jordan, one CTA per matrix).
// lookahead and the next panel run on a side stream while update runs on the
// caller's.  Reads of the panels come from R / Q / D^-1, so the update runs in place
// without races.
// ---------------------------------------------------------------------------
// Block width: 64 for FP32; 32 for FP64, whose per-SM rate on this chip is low
// enough that the serial diagonal-block inverse of each step must stay small.
template <typename T>
struct GJWidth;
template <>
struct GJWidth<float> {
  static constexpr int value = 64;
};
template <>
struct GJWidth<double> {
  static constexpr int value = 32;
};
constexpr int kGJThreads = 256;

struct GJBatch {
  const InvDesc* d;    // per matrix: n, ld, offset into the matrix base
  const int64_t* qoff; // per matrix: offset of its row panels R and Q (NB x ld each)
};

// Inverse of one kb x kb diagonal block by Gauss-Jordan without pivoting (SPD,
// Jacobi-scaled), spread over NW warps (one or two per SM sub-partition): warp w keeps
// rows RW w .. RW w + RW - 1 (RW = NB / NW), lane l the columns l + 32 j.  Per pivot the
// owner warp writes the pivot row twice into double-buffered shared rows, as is
// (column p set to 1) and scaled (a_pc / a_pp, column p 1 / a_pp), one barrier, then
// every thread forms its row factors l_r = a_rp / a_pp (a_rp by shuffle from the lane
// holding column p) and updates each entry with one FMA: a_rc -= l_r a_pc, column p
// from 0 (giving -l_r), row p takes the scaled row.  FP64, whose pipe is the bound on
// this chip, skips the row factor: a_rc -= a_rp (a_pc / a_pp) (column p: -a_rp / a_pp),
// one FMA per entry and no multiply per row.  `src(r, c)` gives the block's
// entries (r, c < kb); beyond kb it is padded with the identity.  Flags in *s_flags:
// DEV_SINGULAR for a non-positive or non-finite pivot, DEV_ILLCOND for a pivot below
// `floor` (Jacobi-scaled matrices have pivots of at most 1).  The inverse goes to Db
// (NB x NB).  Every thread of the first NW warps must call it.
template <typename T, int NB, int NW, typename Src>
__device__ __forceinline__ void gj_diag_body(Src src, int kb, T floor, T* __restrict__ Db, int* s_flags,
                                             T (*prow)[NB], T (*srow)[NB]) {
  constexpr int RW = NB / NW, CJ = NB / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T v[RW][CJ];
#pragma unroll
  for (int i = 0; i < RW; ++i) {
    const int r = RW * warp + i;
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      const int c = lane + 32 * j;
      v[i][j] = (r < kb && c < kb) ? src(r, c) : (r == c ? T(1) : T(0));
    }
  }
  for (int p = 0; p < kb; ++p) {
    const int o = p / RW, sl = p % RW, pl = p & 31, pj = p >> 5;
    T* pr = prow[p & 1];
    T* sc = srow[p & 1];
    if (warp == o) {
      T vp[CJ];
#pragma unroll
      for (int j = 0; j < CJ; ++j) vp[j] = T(0);
#pragma unroll
      for (int i = 0; i < RW; ++i)
        if (i == sl) {
#pragma unroll
          for (int j = 0; j < CJ; ++j) vp[j] = v[i][j];
        }
      T pv = vp[0];
#pragma unroll
      for (int j = 1; j < CJ; ++j)
        if (pj == j) pv = vp[j];
      const T piv = __shfl_sync(0xffffffffu, pv, pl);
      if (lane == 0) {
        if (!(piv > T(0)) || !isfinite(piv))
          *s_flags |= DEV_SINGULAR;
        else if (piv < floor)
          *s_flags |= DEV_ILLCOND;
      }
      const T inv = T(1) / piv;
#pragma unroll
      for (int j = 0; j < CJ; ++j) {
        const int c = lane + 32 * j;
        sc[c] = c == p ? inv : vp[j] * inv;
        pr[c] = c == p ? T(1) : vp[j];
      }
    }
    __syncthreads();
    constexpr bool kRowFactor = sizeof(T) == 4;
    const T inv = sc[p];
    T scl[CJ], m[CJ];
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      scl[j] = sc[lane + 32 * j];
      m[j] = kRowFactor ? pr[lane + 32 * j] : scl[j];
    }
#pragma unroll
    for (int i = 0; i < RW; ++i) {
      const int r = RW * warp + i;
      T a = v[i][0];
#pragma unroll
      for (int j = 1; j < CJ; ++j)
        if (pj == j) a = v[i][j];
      const T l = kRowFactor ? __shfl_sync(0xffffffffu, a, pl) * inv : __shfl_sync(0xffffffffu, a, pl);
#pragma unroll
      for (int j = 0; j < CJ; ++j) {
        const T base_v = (lane + 32 * j == p) ? T(0) : v[i][j];
        const T nv = fma(-l, m[j], base_v);
        v[i][j] = r == p ? scl[j] : nv;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < RW; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) Db[(RW * warp + i) * NB + lane + 32 * j] = v[i][j];
}

// D^-1 of the first diagonal block of every matrix (step 0), read from the matrix
// (row-major, leading dimension ld); later steps fuse it into k_gj_lookahead
template <typename T, int NB>
__global__ void __launch_bounds__(kGJThreads)
k_gj_diag0(GJBatch bt, const T* __restrict__ base, T* __restrict__ Dg, int* status, T floor) {
  const int b = blockIdx.x;
  const InvDesc d = bt.d[b];
  if (d.n <= 0) return;
  const int kb = min(NB, d.n);
  __shared__ T prow[2][NB], srow[2][NB];
  __shared__ int s_flags;
  if (threadIdx.x == 0) s_flags = 0;
  __syncthreads();
  const T* A = base + d.off;
  gj_diag_body<T, NB, kGJThreads / 32>([&](int r, int c) { return A[(int64_t)r * d.ld + c]; }, kb, floor,
                                       Dg + (int64_t)b * NB * NB, &s_flags, prow, srow);
  __syncthreads();
  if (threadIdx.x == 0 && s_flags) atomicOr(status + b, s_flags);
}

// out(NB x CW tile) = sum_l L[i][l] R[l][j], l < kb; thread (tx, ty) of 256 holds
// rows ty + 16 a and columns tx + 16 b
template <typename T, int NB, int CW = NB>
__device__ __forceinline__ void tile_mma(const T (*L)[NB + 1], const T (*R)[CW + 1], int kb,
                                         T acc[NB / 16][CW / 16]) {
  constexpr int RA = NB / 16, RB = CW / 16;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[a][b] = T(0);
  for (int l = 0; l < kb; ++l) {
    T av[RA], bv[RB];
#pragma unroll
    for (int a = 0; a < RA; ++a) av[a] = L[ty + 16 * a][l];
#pragma unroll
    for (int b = 0; b < RB; ++b) bv[b] = R[l][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int b = 0; b < RB; ++b) acc[a][b] += av[a] * bv[b];
  }
}

// Symmetric Gauss-Jordan.  With the blocks before K already processed, the iterate
// is [[X11, X12], [-X12^T, X22]] with X11, X22 symmetric, so every tile below the
// diagonal is +-(the mirrored tile)^T: -1 exactly when one of its two block indices
// is processed.  Only tiles with I <= J are computed; each writes its mirror.
__device__ __forceinline__ int gj_sign(int I, int J, int last_processed) {
  return ((I <= last_processed) != (J <= last_processed)) ? -1 : 1;
}


// old row panel R_Kt = A_Kt and Q_Kt = D^-1 A_Kt: each CTA loads D^-1 once and walks
// `cols` columns (a multiple of the chunk width CW) in chunks, each a register-blocked
// tile product: CW = 64 in FP32 (16 outputs per thread); CW = 16 in FP64, whose few
// FMA per clock per SM favour more, smaller CTAs on the look-ahead path
template <typename T>
struct PanelWidth {
  static constexpr int value = sizeof(T) == 4 ? 64 : 16;
};
template <typename T, int NB>
__global__ void __launch_bounds__(kGJThreads)
k_gj_panel(GJBatch bt, int step, int cols, const T* __restrict__ base, T* __restrict__ R, T* __restrict__ Q,
           const T* __restrict__ Dg) {
  constexpr int CW = PanelWidth<T>::value;
  constexpr int RA = NB / 16, RB = CW / 16;
  const int b = blockIdx.y;
  const InvDesc d = bt.d[b];
  const int k0 = step * NB;
  const int cbase = blockIdx.x * cols;
  if (k0 >= d.n || cbase >= d.n) return;
  const int kb = min(NB, d.n - k0);
  __shared__ T Ds[NB][NB + 1];
  __shared__ T W[NB][CW + 1];
  const T* A = base + d.off;
  const T* Db = Dg + (int64_t)b * NB * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) Ds[e / NB][e % NB] = Db[e];
  T* Rb = R + bt.qoff[b];
  T* Qb = Q + bt.qoff[b];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int c0 = cbase; c0 < min(cbase + cols, d.n); c0 += CW) {
    if (c0 >= k0 && c0 < k0 + NB) continue;   // the diagonal block (uniform across the CTA)
    const int cb = min(CW, d.n - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < NB * CW; e += blockDim.x) {
      const int r = e / CW, c = e % CW;
      T v = T(0);
      if (r < kb && c < cb) {
        v = A[(int64_t)(k0 + r) * d.ld + c0 + c];
        Rb[(int64_t)r * d.ld + c0 + c] = v;
      }
      W[r][c] = v;
    }
    __syncthreads();
    T acc[RA][RB];
    tile_mma<T, NB, CW>(Ds, W, kb, acc);
#pragma unroll
    for (int a = 0; a < RA; ++a) {
      const int r = ty + 16 * a;
#pragma unroll
      for (int c4 = 0; c4 < RB; ++c4) {
        const int c = tx + 16 * c4;
        if (r < kb && c < cb) Qb[(int64_t)r * d.ld + c0 + c] = acc[a][c4];
      }
    }
  }
}

// One tile (I <= J) of the iterate after step K and its mirror: D^-1 (I = J = K),
// the new row panel Q_KJ (I = K), -P_IK D^-1 (J = K) or A_IJ - P_IK Q_KJ.  With `keep`
// (the diagonal tile of step K+1, which only that step's inverse reads) the new values
// go to keep[r][c] instead of the matrix; keep may alias L.
template <typename T, int NB, bool kMirror = true>
__device__ __forceinline__ void gj_tile(const InvDesc& d, int K, int I, int J, T* __restrict__ A,
                                        const T* __restrict__ Db, const T* __restrict__ Rb,
                                        const T* __restrict__ Qb, T (*L)[NB + 1], T (*Rt)[NB + 1],
                                        T (*keep)[NB + 1]) {
  constexpr int RA = NB / 16;
  const int k0 = K * NB;
  const int kb = min(NB, d.n - k0);
  const int i0 = I * NB, j0 = J * NB, ib = min(NB, d.n - i0), jb = min(NB, d.n - j0);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  if (I == K && J == K) {
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x)
      A[(int64_t)(k0 + e / kb) * d.ld + k0 + e % kb] = Db[(e / kb) * NB + e % kb];
    return;
  }
  if (I == K) {
    // new row panel Q_KJ; mirror (J, K) = -Q_KJ^T
    for (int e = threadIdx.x; e < kb * jb; e += blockDim.x) {
      const int r = e / jb, c = e % jb;
      const T v = Qb[(int64_t)r * d.ld + j0 + c];
      A[(int64_t)(k0 + r) * d.ld + j0 + c] = v;
      A[(int64_t)(j0 + c) * d.ld + k0 + r] = -v;
    }
    return;
  }
  // P_IK = s R_KI^T with s = -1 when I is processed (I < K), else +1; the loads run
  // along rows of the panels (coalesced) and transpose through shared memory
  const T sP = I < K ? T(-1) : T(1);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    L[c][r] = (c < ib && r < kb) ? sP * Rb[(int64_t)r * d.ld + i0 + c] : T(0);
    if (J == K)
      Rt[r][c] = (r < kb && c < kb) ? Db[r * NB + c] : T(0);
    else
      Rt[r][c] = (r < kb && c < jb) ? Qb[(int64_t)r * d.ld + j0 + c] : T(0);
  }
  __syncthreads();
  T acc[RA][RA];
  tile_mma<T, NB>(L, Rt, kb, acc);
  if (keep) __syncthreads();   // keep may alias L (uniform branch)
  // tile value: J == K -> -P_IK D^-1, else A_IJ - P_IK Q_KJ;  mirror sign after this step
  const T sM = (T)gj_sign(I, J, K);
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int r = ty + 16 * a;
#pragma unroll
    for (int c4 = 0; c4 < RA; ++c4) {
      const int c = tx + 16 * c4;
      if (r >= ib || c >= jb) continue;
      T* ap = A + (int64_t)(i0 + r) * d.ld + j0 + c;
      const T v = (J == K) ? -acc[a][c4] : (*ap - acc[a][c4]);
      acc[a][c4] = v;
      if (keep)
        keep[r][c] = v;
      else
        *ap = v;
    }
  }
  if (!kMirror || keep || I == J) return;
  // mirror tile (J, I) = sM * tile^T: staged transposed in shared memory, written by rows
  __syncthreads();
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int c4 = 0; c4 < RA; ++c4) L[tx + 16 * c4][ty + 16 * a] = sM * acc[a][c4];
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int c = e / NB, r = e % NB;
    if (c < jb && r < ib) A[(int64_t)(j0 + c) * d.ld + i0 + r] = L[c][r];
  }
}

// Tiles of step K other than block row / column K+1 (one CTA per tile I <= J < nblk;
// the caller may pass fewer blocks than the matrix has, see gj_run).
template <typename T, int NB>
__global__ void __launch_bounds__(kGJThreads)
k_gj_update(GJBatch bt, int step, int nblk, T* __restrict__ base, const T* __restrict__ R, const T* __restrict__ Q,
            const T* __restrict__ Dg) {
  const int b = blockIdx.y;
  const InvDesc d = bt.d[b];
  const int nd = step + 1;
  int t = (int)blockIdx.x, I = 0;
  while (t >= nblk - I) {
    t -= nblk - I;
    ++I;
  }
  const int J = I + t;
  if (I == nd || J == nd) return;
  if (step * NB >= d.n || J * NB >= d.n) return;
  __shared__ T L[NB][NB + 1];
  __shared__ T Rt[NB][NB + 1];
  gj_tile<T, NB>(d, step, I, J, base + d.off, Dg + (int64_t)b * NB * NB, R + bt.qoff[b], Q + bt.qoff[b], L, Rt,
                 nullptr);
}

// Look-ahead launch of step K: the tiles of block row / column K+1 (tile index t takes
// tile (min(K+1, t), max(K+1, t))) up to block column jmax; the CTA of t = K+1 keeps the
// updated diagonal tile in shared memory and inverts it into Dnext, the next step's
// D^-1.  Grid (matrix, tile) with the diagonal tiles in the first grid row, so that
// every matrix's serial inversion starts in the first wave.
template <typename T, int NB>
__global__ void __launch_bounds__(kGJThreads)
k_gj_lookahead(GJBatch bt, int step, int nblk, int jmax, T* __restrict__ base, const T* __restrict__ R,
               const T* __restrict__ Q, const T* __restrict__ Dg, T* __restrict__ Dnext, int* status, T floor) {
  const int b = blockIdx.x;
  const InvDesc d = bt.d[b];
  const int nd = step + 1;
  if (nd >= nblk) return;
  const int y = (int)blockIdx.y;
  const int t = y == 0 ? nd : (y <= nd ? y - 1 : y);
  const int I = min(nd, t), J = max(nd, t);
  if (step * NB >= d.n || J * NB >= d.n || J > jmax) return;
  __shared__ T L[NB][NB + 1];
  __shared__ T Rt[NB][NB + 1];
  __shared__ T prow[2][NB], srow[2][NB];
  __shared__ int s_flags;
  const bool diag = t == nd;
  gj_tile<T, NB>(d, step, I, J, base + d.off, Dg + (int64_t)b * NB * NB, R + bt.qoff[b], Q + bt.qoff[b], L, Rt,
                 diag ? L : nullptr);
  if (!diag) return;
  if (threadIdx.x == 0) s_flags = 0;
  __syncthreads();
  gj_diag_body<T, NB, kGJThreads / 32>([&](int r, int c) { return L[r][c]; }, min(NB, d.n - nd * NB), floor,
                                       Dnext + (int64_t)b * NB * NB, &s_flags, prow, srow);
  __syncthreads();
  if (threadIdx.x == 0 && s_flags) atomicOr(status + b, s_flags);
}

// ---------------------------------------------------------------------------
// FP32 Gauss-Jordan on the tensor cores (3xTF32).
//
// The same symmetric blocked Gauss-Jordan as above (block width 64), with every block
// contraction on the tensor cores.  At step K, for every tile (I <= J) outside block
// row / column K+1,
//   A_IJ <- [J == K ? 0 : A_IJ] - s_I G_IJ,   G = R_K^T Q'_K,
// with R_K the old row panel, Q'_K = D^-1 R_K except in block column K, where it is
// D^-1 itself, and s_I = -1 for a processed block (I < K), +1 otherwise (the iterate is
// [[X11, X12], [-X12^T, X22]], so P_IK = s_I R_KI^T); block row K takes Q'_K, and each
// tile above the diagonal also writes its mirror.  G is a 64-deep contraction per
// output tile: tcgen05.mma kind::tf32 with each FP32 operand split into hi = rn_tf32(x)
// and lo = rn_tf32(x - hi) and three products lo.hi + hi.lo + hi.hi accumulated in
// FP32 in tensor memory (the 3xTF32 split product, about FP32 accuracy).  Three
// launches per step: the update (k_gj_update_tc) on the caller's stream; on a side
// stream block row K+1 with the next diagonal inverse (k_gj_row_tc) and the next row
// panel Q_{K+1} = D^-1 R_{K+1} (k_gj_qpanel_tc), both as transposed tensor-core tiles.
//
// Operands live in global memory as K-major split images, written once per step by
// the kernel that produces them: plane p of image b holds rows (matrix columns) x 32
// floats, planes {hi k 0-31, hi k 32-63, lo k 0-31, lo k 32-63}; zeros beyond the
// block's kb rows.  A CTA loads a 128-row slab of one image and a 64-row slab of
// another with two TMA tensor copies (128-byte swizzle), which is the canonical K-major
// SW128 operand layout of the MMA.  One CTA per 128 x 64 output tile, eight warps:
// warp 0 allocates 64 tensor-memory columns, one thread issues the copies and the 24
// MMAs, and warps w and w + 4 read back the accumulator lanes 32 (w % 4) .. + 31 (one
// row each) in two column halves with tcgen05.ld.
// ---------------------------------------------------------------------------
constexpr int kTcM = 128, kTcN = 64, kTcThreads = 256;
constexpr int kTcPlaneA = kTcM * 128, kTcPlaneB = kTcN * 128;   // bytes per operand plane
constexpr int kTcSmem = 4 * kTcPlaneA + 4 * kTcPlaneB;           // 96 KB
constexpr unsigned long long kTcWaitNs = 1000000000ull;          // bounded waits: one second

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long tc_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool tc_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(tc_smem(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase of the given parity, bounded by kTcWaitNs; false on expiry
__device__ bool tc_wait(uint64_t* bar, unsigned parity) {
  if (tc_try_wait(bar, parity)) return true;
  const unsigned long long t0 = tc_now();
  while (!tc_try_wait(bar, parity))
    if (tc_now() - t0 > kTcWaitNs) return false;
  return true;
}
// K-major operand with 128-byte swizzle (8-row groups 1024 bytes apart), SM100 descriptor
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// kind::tf32, D FP32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ float tc_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// write the K-major split images of one 64-column panel chunk, image rows c0 .. c0 + 63:
// v(k, c) for k < kb and c < cb, zero elsewhere (so the rows of a matrix's last chunk
// beyond its size hold zeros)
template <typename F>
__device__ __forceinline__ void tc_write_image(float* __restrict__ img, int rows_pad, int c0, int cb, int kb, F v) {
  const int64_t plane = (int64_t)rows_pad * 32;
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int c = e >> 6, k = e & 63;
    const float x = (k < kb && c < cb) ? v(k, c) : 0.f;
    const float hi = tc_tf32(x);
    const float lo = tc_tf32(x - hi);
    const int64_t o = (int64_t)(c0 + c) * 32 + (k & 31);
    img[(k >> 5) * plane + o] = hi;
    img[(2 + (k >> 5)) * plane + o] = lo;
  }
}

struct TcImages {
  float* R;        // [2 parities][batch][4 planes][rows_pad][32]
  float* Q;
  int rows_pad;
  int nb;          // matrices in the batch
};

// old row panel R = A_K*, Q = D^-1 A_K* (as k_gj_panel) plus their split images for the
// tensor-core update; the CTA of the diagonal chunk writes the image of D^-1 (block
// column K of Q')
__global__ void __launch_bounds__(kGJThreads)
k_gj_panel_tc(GJBatch bt, int step, const float* __restrict__ base, float* __restrict__ R, float* __restrict__ Q,
              const float* __restrict__ Dg, TcImages im) {
  constexpr int NB = 64, CW = 64, RA = NB / 16, RB = CW / 16;
  const int b = blockIdx.y;
  const InvDesc d = bt.d[b];
  const int k0 = step * NB;
  const int c0 = blockIdx.x * CW;
  if (k0 >= d.n || c0 >= d.n) return;
  const int kb = min(NB, d.n - k0), cb = min(CW, d.n - c0);
  __shared__ float Ds[NB][NB + 1];
  __shared__ float W[NB][CW + 1];
  const float* Db = Dg + (int64_t)b * NB * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) Ds[e / NB][e % NB] = Db[e];
  const int par = step & 1;
  const int64_t img_off = ((int64_t)par * im.nb + b) * 4 * im.rows_pad * 32;
  __syncthreads();
  if (c0 == k0) {   // diagonal chunk: Q' = D^-1, R unused (block row K takes Q'); uniform across the CTA
    tc_write_image(im.Q + img_off, im.rows_pad, c0, cb, kb, [&](int k, int c) { return Ds[k][c]; });
    tc_write_image(im.R + img_off, im.rows_pad, c0, 0, 0, [&](int, int) { return 0.f; });
    return;
  }
  const float* A = base + d.off;
  float* Rb = R + bt.qoff[b];
  float* Qb = Q + bt.qoff[b];
  for (int e = threadIdx.x; e < NB * CW; e += blockDim.x) {
    const int r = e / CW, c = e % CW;
    float v = 0.f;
    if (r < kb && c < cb) {
      v = A[(int64_t)(k0 + r) * d.ld + c0 + c];
      Rb[(int64_t)r * d.ld + c0 + c] = v;
    }
    W[r][c] = v;
  }
  __syncthreads();
  tc_write_image(im.R + img_off, im.rows_pad, c0, cb, kb, [&](int k, int c) { return W[k][c]; });
  float acc[RA][RB];
  tile_mma<float, NB, CW>(Ds, W, kb, acc);
  __syncthreads();   // W is reused for Q
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int r = ty + 16 * a;
#pragma unroll
    for (int c4 = 0; c4 < RB; ++c4) {
      const int c = tx + 16 * c4;
      W[r][c] = acc[a][c4];
      if (r < kb && c < cb) Qb[(int64_t)r * d.ld + c0 + c] = acc[a][c4];
    }
  }
  __syncthreads();
  tc_write_image(im.Q + img_off, im.rows_pad, c0, cb, kb, [&](int k, int c) { return W[k][c]; });
}

// ---- shared pieces of the tensor-core tile kernels (128 threads, one 128 x 64 FP32
// accumulator in 64 tensor-memory columns; operand A = 4 planes x 128 image rows, operand
// B = 4 planes x 64 image rows, both staged by TMA into dynamic shared memory) ----
struct TcShared {
  uint64_t bar_load, bar_mma;
  uint32_t tmem;
};

// barriers and the accumulator's tensor memory (warp 0 allocates); every thread calls it
__device__ __forceinline__ uint32_t tc_begin(TcShared& ts) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&ts.bar_load)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&ts.bar_mma)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&ts.tmem)),
                 "r"(kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return ts.tmem;
}

// releases the tensor memory once every thread is done with it; every thread calls it
__device__ __forceinline__ void tc_end(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN) : "memory");
  }
}

// D[m][n] = sum_k A[m][k] B[n][k] over the 64 k of the images (3xTF32): thread 0 loads
// operand A (rows ra.. of image ia through mA) and operand B (rows rb.. of image ib
// through mB) and issues the 24 MMAs; every thread waits for the accumulator.  Returns
// false (same value in every thread) after a wait expired: DEV_TIMEOUT is recorded and
// the copies or products in flight are waited for (bounded) before returning.
__device__ bool tc_tile(TcShared& ts, unsigned char* sA, unsigned char* sB, const CUtensorMap* mA, int ra, int ia,
                        const CUtensorMap* mB, int rb, int ib, uint32_t tmem, int* flag) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(&ts.bar_load)),
                 "r"((unsigned)kTcSmem)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(tc_smem(sA)),
        "l"(reinterpret_cast<uint64_t>(mA)), "r"(0), "r"(ra), "r"(0), "r"(ia), "r"(tc_smem(&ts.bar_load))
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(tc_smem(sB)),
        "l"(reinterpret_cast<uint64_t>(mB)), "r"(0), "r"(rb), "r"(0), "r"(ib), "r"(tc_smem(&ts.bar_load))
        : "memory");
  }
  bool ok = tc_wait(&ts.bar_load, 0);
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) {
      atomicOr(flag, DEV_TIMEOUT);
      tc_wait(&ts.bar_load, 0);
    }
    return false;
  }
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t a0 = tc_smem(sA), b0 = tc_smem(sB);
    uint32_t acc = 0;
    // planes: 0 hi k 0-31, 1 hi k 32-63, 2 lo k 0-31, 3 lo k 32-63; products lo.hi, hi.lo, hi.hi
#pragma unroll
    for (int prod = 0; prod < 3; ++prod)
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int pa = prod == 0 ? 2 : 0, pb = prod == 1 ? 2 : 0;
        const uint32_t off = (uint32_t)((kk & 3) * 32);
        const uint32_t aa = a0 + (uint32_t)((pa + (kk >> 2)) * kTcPlaneA) + off;
        const uint32_t bb = b0 + (uint32_t)((pb + (kk >> 2)) * kTcPlaneB) + off;
        tc_mma(tmem, tc_desc(aa), tc_desc(bb), acc);
        acc = 1;
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc_smem(&ts.bar_mma))
                 : "memory");
  }
  ok = tc_wait(&ts.bar_mma, 0);
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) {
      atomicOr(flag, DEV_TIMEOUT);
      tc_wait(&ts.bar_mma, 0);
    }
    return false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

// accumulator columns c .. c+15 of this thread's row (TMEM lane 32 (warp % 4) + lane: warps w
// and w + 4 share the lanes of one quarter and take different columns); warp-collective
__device__ __forceinline__ void tc_ld16(uint32_t tmem, int c, float v[16]) {
  uint32_t r[16];
  const uint32_t taddr = tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + (uint32_t)c;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// 16 consecutive k (k0 .. k0+15, k0 a multiple of 16) of one image row: split and stored
// into the hi and lo planes
__device__ __forceinline__ void tc_store_split16(float* __restrict__ img, int rows_pad, int row, int k0,
                                                 const float v[16]) {
  const int64_t plane = (int64_t)rows_pad * 32;
  float* hi = img + (k0 >> 5) * plane + (int64_t)row * 32 + (k0 & 31);
  float* lo = hi + 2 * plane;
#pragma unroll
  for (int q = 0; q < 16; q += 4) {
    float h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      h[t] = tc_tf32(v[q + t]);
      l[t] = tc_tf32(v[q + t] - h[t]);
    }
    *reinterpret_cast<float4*>(hi + q) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + q) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

__device__ __forceinline__ unsigned char* tc_dynamic_smem() {
  extern __shared__ __align__(1024) unsigned char tc_dyn[];
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_dyn) + 1023) & ~(uintptr_t)1023);
}

struct TcMaps {
  CUtensorMap R128, Q64, Q128, R64, D64;
};

// Block row K+1 of step K on the tensor cores, transposed: for the 128 columns j of this
// CTA, D[j][i] = sum_k Q'_K[k][j] R_K[k][k1 + i] = G[k1 + i][j] (operand A = the Q' image,
// operand B = the R image rows of block K+1), and A[k1 + i][j] <- [j in K ? 0 : A] - G
// (s = +1: block K+1 is unprocessed), and its mirror A[j][k1 + i] = sM A[k1 + i][j] (block
// column K+1, not read by the update).  Thread (m, h): column j = j0 + m, rows i of half h;
// the old values are loaded before the operands arrive.  Each thread also writes its
// half of row j of the next step's R image; the CTA holding block column K+1 keeps that
// 64 x 64 tile in shared memory (over the freed operand buffers), inverts it into Dnext
// (SIMT Gauss-Jordan) and writes the split image of Dnext.
__global__ void __launch_bounds__(kTcThreads)
k_gj_row_tc(GJBatch bt, int step, float* __restrict__ base, float* __restrict__ Dnext, int* status, float floor,
            const __grid_constant__ TcMaps maps, TcImages im, float* __restrict__ Dimg) {
  constexpr int NB = 64;
  const int b = blockIdx.y;
  const InvDesc d = bt.d[b];
  const int n = d.n, k0 = step * NB, k1 = k0 + NB;
  const int j0 = blockIdx.x * kTcM;
  if (k1 >= n || j0 >= n) return;
  const int kb1 = min(NB, n - k1);
  unsigned char* smem = tc_dynamic_smem();
  __shared__ TcShared ts;
  __shared__ float prow[2][NB], srow[2][NB];
  __shared__ int s_flags;
  const int m = threadIdx.x & 127, h = threadIdx.x >> 7;   // h: rows 32 h .. 32 h + 31 of block K+1
  const int j = j0 + ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31);
  (void)m;
  const bool colok = j < n;
  const bool colK = j >= k0 && j < k1;
  const bool diagc = j >= k1 && j < k1 + NB;
  float* Acol = base + d.off + (int64_t)k1 * d.ld + j;
  float old[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int i = 32 * h + q;
    old[q] = (colok && !colK && i < kb1) ? Acol[(int64_t)i * d.ld] : 0.f;
  }
  const uint32_t tmem = tc_begin(ts);
  const int img_cur = (step & 1) * im.nb + b, img_next = ((step + 1) & 1) * im.nb + b;
  const bool ok = tc_tile(ts, smem, smem + 4 * kTcPlaneA, &maps.Q128, j0, img_cur, &maps.R64, k1, img_cur, tmem,
                          status + b);
  const bool has_diag = k1 >= j0 && k1 < j0 + kTcM;
  float (*T)[NB + 1] = reinterpret_cast<float (*)[NB + 1]>(smem);   // the operands are consumed
  if (ok) {
    float* imgR = im.R + (int64_t)img_next * 4 * im.rows_pad * 32;
#pragma unroll
    for (int cc = 0; cc < 32; cc += 16) {
      float g[16];
      tc_ld16(tmem, 32 * h + cc, g);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = 32 * h + cc + q;
        float v = 0.f;
        if (colok && i < kb1) {
          v = old[cc + q] - g[q];
          Acol[(int64_t)i * d.ld] = v;
        }
        g[q] = v;
        if (diagc) T[i][j - k1] = v;
      }
      // mirror into block column K+1: A[j][k1 + i] = sM A[k1 + i][j], 16 consecutive values
      if (colok && !diagc) {
        const float sM = (float)gj_sign(j / NB, step + 1, step);
        float* mrow = base + d.off + (int64_t)j * d.ld + k1 + 32 * h + cc;
#pragma unroll
        for (int q4 = 0; q4 < 16; q4 += 4) {
          const int i = 32 * h + cc + q4;   // kb1 is a multiple of 4 unless block K+1 is the last
          if (i + 3 < kb1) {
            *reinterpret_cast<float4*>(mrow + q4) =
                make_float4(sM * g[q4], sM * g[q4 + 1], sM * g[q4 + 2], sM * g[q4 + 3]);
          } else {
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (i + t < kb1) mrow[q4 + t] = sM * g[q4 + t];
          }
        }
      }
      tc_store_split16(imgR, im.rows_pad, j, 32 * h + cc, g);
    }
  }
  if (ok && has_diag) {
    if (threadIdx.x == 0) s_flags = 0;
    __syncthreads();
    float* Dn = Dnext + (int64_t)b * NB * NB;
    gj_diag_body<float, NB, kTcThreads / 32>([&](int r, int c) { return T[r][c]; }, kb1, floor, Dn, &s_flags, prow,
                                             srow);
    __syncthreads();
    if (threadIdx.x == 0 && s_flags) atomicOr(status + b, s_flags);
    // split image of D^-1 (rows k, 64 k' each; zeros outside the kb1 x kb1 block)
    float* imgD = Dimg + (int64_t)img_next * 4 * NB * 32;
    {
      const int r = threadIdx.x >> 2, c0 = (threadIdx.x & 3) * 16;
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = (r < kb1 && c0 + q < kb1) ? Dn[r * NB + c0 + q] : 0.f;
      tc_store_split16(imgD, NB, r, c0, v);
    }
  }
  tc_end(tmem);
}

// Row panel of step K+1 on the tensor cores, transposed: for the 128 columns j of this
// CTA, D[j][k] = sum_l R_{K+1}[l][j] D^-1[k][l] = Q_{K+1}[k][j] (operand A = the R image,
// operand B = the image of D^-1).  Each thread (one column) writes Q_{K+1}[., j] and row j
// of the Q' image (D^-1 itself in block column K+1).
__global__ void __launch_bounds__(kTcThreads)
k_gj_qpanel_tc(GJBatch bt, int step1, float* __restrict__ Q, const float* __restrict__ Dg, int* status,
               const __grid_constant__ TcMaps maps, TcImages im) {
  constexpr int NB = 64;
  const int b = blockIdx.y;
  const InvDesc d = bt.d[b];
  const int n = d.n, k0 = step1 * NB;
  const int j0 = blockIdx.x * kTcM;
  if (k0 >= n || j0 >= n) return;
  const int kb = min(NB, n - k0);
  unsigned char* smem = tc_dynamic_smem();
  __shared__ TcShared ts;
  const uint32_t tmem = tc_begin(ts);
  const int img = (step1 & 1) * im.nb + b;
  const bool ok =
      tc_tile(ts, smem, smem + 4 * kTcPlaneA, &maps.R128, j0, img, &maps.D64, 0, img, tmem, status + b);
  if (ok) {
    const int h = threadIdx.x >> 7;   // rows k of half h
    const int j = j0 + ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31);
    const bool colok = j < n;
    const bool diagc = j >= k0 && j < k0 + NB;
    const float* Db = Dg + (int64_t)b * NB * NB;
    float* Qcol = Q + bt.qoff[b] + j;
    float* imgQ = im.Q + (int64_t)img * 4 * im.rows_pad * 32;
#pragma unroll
    for (int cc = 32 * h; cc < 32 * h + 32; cc += 16) {
      float g[16];
      tc_ld16(tmem, cc, g);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int k = cc + q;
        float v = 0.f;
        if (colok && k < kb) {
          v = g[q];
          Qcol[(int64_t)k * d.ld] = v;
          if (diagc) v = (j - k0 < kb) ? Db[k * NB + (j - k0)] : 0.f;
        }
        g[q] = v;
      }
      tc_store_split16(imgQ, im.rows_pad, j, cc, g);
    }
  }
  tc_end(tmem);
}

// Tensor-core update of step K: one CTA per 128 x 64 tile (rows i0.., column block J) of
// one matrix with J >= the first row block of the tile (upper triangle).  Rows of block
// <= J are updated (block row K takes Q'_K); rows of block < J also write the mirror
// A_ji = sM A_ij (sM = -1 when exactly one of the two blocks is processed after step K),
// so the lower triangle is written without being read.  Block row and column K+1 are the
// row kernel's.
__global__ void __launch_bounds__(kTcThreads)
k_gj_update_tc(GJBatch bt, int step, int tiles_n, float* __restrict__ base, const float* __restrict__ Q,
               const float* __restrict__ Dg, int* status, const __grid_constant__ TcMaps maps, int nb) {
  constexpr int NB = 64;
  const int b = blockIdx.y;
  const InvDesc d = bt.d[b];
  const int n = d.n, k0 = step * NB, k1 = k0 + NB;
  const int i0 = (blockIdx.x / tiles_n) * kTcM, j0 = (blockIdx.x % tiles_n) * kTcN;
  const int J = j0 / NB, blk0 = i0 / NB;
  if (k0 >= n || i0 >= n || j0 >= n || J < blk0 || J == step + 1) return;
  // rows updated here: block rows blk0, blk0 + 1 that are <= J and not K+1
  const bool work0 = blk0 != step + 1, work1 = (blk0 + 1) * NB < n && blk0 + 1 <= J && blk0 + 1 != step + 1;
  if (!work0 && !work1) return;
  unsigned char* smem = tc_dynamic_smem();
  __shared__ TcShared ts;
  // thread (row m, half h): row i = i0 + m, columns j0 + 32 h .. j0 + 32 h + 31; the old
  // values (or, in block row K, Q'_K) are loaded before the operands arrive
  const int h = threadIdx.x >> 7;
  const int i = i0 + ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31);
  const int bi = i / NB;
  const bool row_ok = i < n && bi != step + 1 && bi <= J;
  const float s = bi < step ? -1.f : 1.f;
  const float sM = (float)gj_sign(bi, J, step);
  float* Arow = base + d.off + (int64_t)i * d.ld;
  const int jh = j0 + 32 * h;
  float old[32];
#pragma unroll
  for (int g4 = 0; g4 < 8; ++g4) {
    const int j = jh + 4 * g4;   // first column of this group of four (16-byte aligned)
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row_ok && j < n) v = *reinterpret_cast<const float4*>(Arow + j);
    old[4 * g4] = v.x;
    old[4 * g4 + 1] = v.y;
    old[4 * g4 + 2] = v.z;
    old[4 * g4 + 3] = v.w;
  }
  if (row_ok && bi == step) {
    const float* Qrow = Q + bt.qoff[b] + (int64_t)(i - k0) * d.ld;
    const float* Drow = Dg + (int64_t)b * NB * NB + (int64_t)(i - k0) * NB;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int jj = jh + q;
      if (jj < n) old[q] = (jj >= k0 && jj < k1) ? Drow[jj - k0] : Qrow[jj];
    }
  }
  const uint32_t tmem = tc_begin(ts);
  const int img = (step & 1) * nb + b;   // images of this step's parity
  const bool ok = tc_tile(ts, smem, smem + 4 * kTcPlaneA, &maps.R128, i0, img, &maps.Q64, j0, img, tmem, status + b);
  if (ok) {
    const bool mirror = row_ok && bi < J;
#pragma unroll
    for (int cc = 0; cc < 32; cc += 16) {
      float g[16];
      tc_ld16(tmem, 32 * h + cc, g);
      if (!row_ok) continue;
#pragma unroll
      for (int g4 = 0; g4 < 4; ++g4) {
        const int j = jh + cc + 4 * g4;
        if (j >= n) continue;             // the group lies in the row's padding or beyond
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int jj = j + q;
          const float o = old[cc + 4 * g4 + q];
          if (jj >= n || bi == step)
            v[q] = o;                     // padding keeps its (zero) value; block row K takes Q'_K
          else
            v[q] = ((jj >= k0 && jj < k1) ? 0.f : o) - s * g[4 * g4 + q];
        }
        *reinterpret_cast<float4*>(Arow + j) = make_float4(v[0], v[1], v[2], v[3]);
        if (mirror) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (j + q < n) base[d.off + (int64_t)(j + q) * d.ld + i] = sM * v[q];
        }
      }
    }
  }
  tc_end(tmem);
}

// cuTensorMapEncodeTiled from the driver (looked up once)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::mutex mu;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    UFE_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    UFE_REQUIRE(p && q == cudaDriverEntryPointSuccess, UFE_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 4-D map over an image arena [2 nb][4][rows_pad][32] floats, box {32, box_rows, 4, 1}
static CUtensorMap image_map(float* arena, int rows_pad, int nb, int box_rows) {
  CUtensorMap tm;
  const cuuint64_t dims[4] = {32, (cuuint64_t)rows_pad, 4, (cuuint64_t)(2 * nb)};
  const cuuint64_t strides[3] = {128, (cuuint64_t)rows_pad * 128, (cuuint64_t)rows_pad * 512};
  const cuuint32_t box[4] = {32, (cuuint32_t)box_rows, 4, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = tensor_map_encoder()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, arena, dims, strides, box, es,
                                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  UFE_REQUIRE(r == CUDA_SUCCESS, UFE_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return tm;
}

// library-owned side stream of the current device (look-ahead of the Gauss-Jordan steps)
static cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t st[128] = {};
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
  std::lock_guard<std::mutex> lock(mu);
  if (!st[dev]) UFE_CUDA(cudaStreamCreateWithFlags(&st[dev], cudaStreamNonBlocking));
  return st[dev];
}

struct GJEvents {
  cudaEvent_t e[2] = {nullptr, nullptr};
  GJEvents() {
    for (auto& x : e) UFE_CUDA(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
  }
  ~GJEvents() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
  cudaEvent_t operator[](int i) const { return e[i]; }
};

// Envelope of a symmetric matrix under block Gauss-Jordan.  With f_j the first column
// holding a nonzero in row j, the unprocessed part keeps its envelope (as in a Cholesky
// factorisation: no fill left of f_j), and a processed row reaches an unprocessed
// column j only through rows whose envelope starts in the processed columns.  So at
// step K block column K (and, by symmetry, block row K) is zero below (right of) block
// lim_K = max{ j : f_j <= last column of block K } / NB, every update of step K stays
// inside blocks [0, lim_K]^2, and lim_K is nondecreasing with lim_K >= K.
static std::vector<int> gj_envelope(const std::vector<int32_t>& first_col, int n, int NB) {
  const int nblk = (n + NB - 1) / NB;
  std::vector<int> reach(nblk, 0);   // reach[b] = the largest row j whose envelope starts in block b
  for (int j = 0; j < n; ++j) {
    const int b = std::min(std::max(first_col[j], 0), j) / NB;
    reach[b] = std::max(reach[b], j);
  }
  std::vector<int> lim(nblk);
  int r = 0;
  for (int K = 0; K < nblk; ++K) {
    r = std::max(r, reach[K]);
    lim[K] = std::max(K, r / NB);
  }
  return lim;
}

// lim (optional): per step K the last block that step K touches (gj_envelope); without
// it every step covers the whole matrix
template <typename T>
static void gj_run(const std::vector<InvDesc>& descs, T* base, int* status, cudaStream_t s, T floor,
                   const std::vector<int>* lim = nullptr) {
  constexpr int NB = GJWidth<T>::value;
  if (descs.empty()) return;
  int nmax = 0;
  std::vector<int64_t> qoff(descs.size());
  int64_t nq = 0;
  for (size_t b = 0; b < descs.size(); ++b) {
    nmax = std::max(nmax, descs[b].n);
    qoff[b] = nq;
    nq += (int64_t)NB * descs[b].ld;
  }
  if (nmax == 0) return;
  DBuf<InvDesc> dd;
  DBuf<int64_t> dq;
  DBuf<T> R, Q, D;
  dd.alloc(descs.size(), s);
  dq.alloc(descs.size(), s);
  R.alloc(2 * std::max<int64_t>(nq, 1), s);   // panels of two consecutive steps (look-ahead)
  Q.alloc(2 * std::max<int64_t>(nq, 1), s);
  nq = std::max<int64_t>(nq, 1);
  cudaStream_t s2 = side_stream();
  GJEvents ev;
  D.alloc(2 * descs.size() * NB * NB, s);
  T* Dbuf[2] = {D.p, D.p + descs.size() * NB * NB};
  UFE_CUDA(cudaMemcpyAsync(dd.p, descs.data(), descs.size() * sizeof(InvDesc), cudaMemcpyHostToDevice, s));
  UFE_CUDA(cudaMemcpyAsync(dq.p, qoff.data(), qoff.size() * 8, cudaMemcpyHostToDevice, s));
  const GJBatch bt{dd.p, dq.p};
  const int nblk = (nmax + NB - 1) / NB;
  const unsigned nb = (unsigned)descs.size();
  UFE_REQUIRE(!lim || (descs.size() == 1 && (int)lim->size() == nblk), UFE_ERR_INVALID_ARG,
              "an envelope applies to one matrix, one entry per block");
  auto last = [&](int step) { return lim ? (*lim)[step] : nblk - 1; };
  // columns of the row panel of a step: its envelope and, for the look-ahead, block K+2
  auto panel_blocks = [&](int step) {
    return (unsigned)((std::min(nmax, (std::min(std::max(last(step), step + 1), nblk - 1) + 1) * NB) +
                       PanelWidth<T>::value - 1) /
                      PanelWidth<T>::value);
  };
  const int pcols = PanelWidth<T>::value;   // one chunk per CTA
  {
    TimedLaunch tl;
    tl.begin(sizeof(T) == 8 ? "gj_diag_f64" : "gj_diag_f32", s);
    k_gj_diag0<T, NB><<<nb, kGJThreads, 0, s>>>(bt, base, Dbuf[0], status, floor);
    UFE_CHECK_LAUNCH();
    tl.end(s);
  }
  for (int step = 0; step < nblk; ++step) {
    T* Dc = Dbuf[step & 1];
    T* Dn = Dbuf[(step + 1) & 1];
    T* Rc = R.p + (step & 1) * nq;
    T* Qc = Q.p + (step & 1) * nq;
    if (step == 0) {
      k_gj_panel<T, NB><<<dim3(panel_blocks(0), nb), kGJThreads, 0, s>>>(bt, 0, pcols, base, Rc, Qc, Dc);
      UFE_CHECK_LAUNCH();
    }
    // look-ahead: block row / column K+1 with the next diagonal inverse, then the next
    // panel, on the side stream while the main stream updates the other tiles
    UFE_CUDA(cudaEventRecord(ev[0], s));
    UFE_CUDA(cudaStreamWaitEvent(s2, ev[0], 0));
    if (step + 1 < nblk) {
      T* Rn = R.p + ((step + 1) & 1) * nq;
      T* Qn = Q.p + ((step + 1) & 1) * nq;
      TimedLaunch ta;
      ta.begin(sizeof(T) == 8 ? "gj_lookahead_f64" : "gj_lookahead_f32", s2);
      const int jmax = std::max(last(step), step + 1);
      k_gj_lookahead<T, NB><<<dim3(nb, jmax + 1), kGJThreads, 0, s2>>>(bt, step, nblk, jmax, base, Rc, Qc, Dc, Dn,
                                                                       status, floor);
      UFE_CHECK_LAUNCH();
      ta.end(s2);
      TimedLaunch tp;
      tp.begin(sizeof(T) == 8 ? "gj_panel_f64" : "gj_panel_f32", s2);
      k_gj_panel<T, NB><<<dim3(panel_blocks(step + 1), nb), kGJThreads, 0, s2>>>(bt, step + 1, pcols, base, Rn, Qn,
                                                                                 Dn);
      UFE_CHECK_LAUNCH();
      tp.end(s2);
    }
    TimedLaunch tl;
    tl.begin(sizeof(T) == 8 ? "gj_update_f64" : "gj_update_f32", s);
    const int nl = last(step) + 1;
    k_gj_update<T, NB><<<dim3((unsigned)(nl * (nl + 1) / 2), nb), kGJThreads, 0, s>>>(bt, step, nl, base, Rc, Qc, Dc);
    UFE_CHECK_LAUNCH();
    tl.end(s);
    UFE_CUDA(cudaEventRecord(ev[1], s2));
    UFE_CUDA(cudaStreamWaitEvent(s, ev[1], 0));
  }
}

// FP32 batched inversion with the tensor-core update (same step structure as gj_run:
// update on the caller's stream, look-ahead and next panel on the side stream)
static void gj_run_tc(const std::vector<InvDesc>& descs, float* base, int* status, cudaStream_t s, float floor) {
  constexpr int NB = 64;
  if (descs.empty()) return;
  int nmax = 0;
  std::vector<int64_t> qoff(descs.size());
  int64_t nq = 0;
  for (size_t b = 0; b < descs.size(); ++b) {
    nmax = std::max(nmax, descs[b].n);
    qoff[b] = nq;
    nq += (int64_t)NB * descs[b].ld;
  }
  if (nmax == 0) return;
  nq = std::max<int64_t>(nq, 1);
  const int nb = (int)descs.size();
  const int rows_pad = (nmax + kTcM - 1) / kTcM * kTcM;
  DBuf<InvDesc> dd;
  DBuf<int64_t> dq;
  DBuf<float> R, Q, D, imR, imQ, imD;
  dd.alloc(descs.size(), s);
  dq.alloc(descs.size(), s);
  R.alloc(nq, s);   // the step-0 panel's raw R (the later steps keep R only as an image)
  Q.alloc(2 * nq, s);
  D.alloc(2 * (int64_t)nb * NB * NB, s);
  const int64_t img = 2 * (int64_t)nb * 4 * rows_pad * 32;
  imR.alloc(img, s);
  imQ.alloc(img, s);
  imD.alloc(2 * (int64_t)nb * 4 * NB * 32, s);
  UFE_CUDA(cudaMemcpyAsync(dd.p, descs.data(), descs.size() * sizeof(InvDesc), cudaMemcpyHostToDevice, s));
  UFE_CUDA(cudaMemcpyAsync(dq.p, qoff.data(), qoff.size() * 8, cudaMemcpyHostToDevice, s));
  TcMaps maps;
  maps.R128 = image_map(imR.p, rows_pad, nb, kTcM);
  maps.R64 = image_map(imR.p, rows_pad, nb, kTcN);
  maps.Q128 = image_map(imQ.p, rows_pad, nb, kTcM);
  maps.Q64 = image_map(imQ.p, rows_pad, nb, kTcN);
  maps.D64 = image_map(imD.p, NB, nb, kTcN);
  {
    static std::mutex mu;
    static bool done[128] = {};
    int dev = 0;
    UFE_CUDA(cudaGetDevice(&dev));
    UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
      UFE_CUDA(cudaFuncSetAttribute(k_gj_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem + 1024));
      UFE_CUDA(cudaFuncSetAttribute(k_gj_row_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem + 1024));
      UFE_CUDA(cudaFuncSetAttribute(k_gj_qpanel_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem + 1024));
      done[dev] = true;
    }
  }
  const TcImages im{imR.p, imQ.p, rows_pad, nb};
  const GJBatch bt{dd.p, dq.p};
  const int nblk = (nmax + NB - 1) / NB;
  const int tiles_n = (nmax + kTcN - 1) / kTcN, tiles_m = rows_pad / kTcM;
  cudaStream_t s2 = side_stream();
  GJEvents ev;
  float* Dbuf[2] = {D.p, D.p + (int64_t)nb * NB * NB};
  {
    TimedLaunch tl;
    tl.begin("gj_diag_f32", s);
    k_gj_diag0<float, NB><<<nb, kGJThreads, 0, s>>>(bt, base, Dbuf[0], status, floor);
    UFE_CHECK_LAUNCH();
    tl.end(s);
  }
  // step 0's panel and images (SIMT: R from the matrix, Q = D^-1 R)
  k_gj_panel_tc<<<dim3((unsigned)((nmax + NB - 1) / NB), nb), kGJThreads, 0, s>>>(bt, 0, base, R.p, Q.p, Dbuf[0],
                                                                                  im);
  UFE_CHECK_LAUNCH();
  const size_t dyn = kTcSmem + 1024;
  for (int step = 0; step < nblk; ++step) {
    UFE_CUDA(cudaEventRecord(ev[0], s));
    UFE_CUDA(cudaStreamWaitEvent(s2, ev[0], 0));
    if (step + 1 < nblk) {
      // side stream: block row K+1 and the next diagonal inverse, then the next panel
      TimedLaunch ta;
      ta.begin("gj_lookahead_f32", s2);
      k_gj_row_tc<<<dim3(tiles_m, nb), kTcThreads, dyn, s2>>>(bt, step, base, Dbuf[(step + 1) & 1], status, floor,
                                                              maps, im, imD.p);
      UFE_CHECK_LAUNCH();
      ta.end(s2);
      TimedLaunch tp;
      tp.begin("gj_panel_f32", s2);
      k_gj_qpanel_tc<<<dim3(tiles_m, nb), kTcThreads, dyn, s2>>>(bt, step + 1, Q.p + ((step + 1) & 1) * nq,
                                                                 Dbuf[(step + 1) & 1], status, maps, im);
      UFE_CHECK_LAUNCH();
      tp.end(s2);
    }
    TimedLaunch tl;
    tl.begin("gj_update_f32", s);
    k_gj_update_tc<<<dim3(tiles_m * tiles_n, nb), kTcThreads, dyn, s>>>(bt, step, tiles_n, base,
                                                                        Q.p + (step & 1) * nq, Dbuf[step & 1],
                                                                        status, maps, nb);
    UFE_CHECK_LAUNCH();
    tl.end(s);
    UFE_CUDA(cudaEventRecord(ev[1], s2));
    UFE_CUDA(cudaStreamWaitEvent(s, ev[1], 0));
  }
}

bool fp32_tensor_cores() {
  const char* e = getenv("UFE_FP32_GJ");
  return !(e && std::string(e) == "simt");
}

template <typename T>
void batched_inverse(const std::vector<InvDesc>& descs, T* base, int* status, cudaStream_t s, T pivot_floor) {
  if constexpr (sizeof(T) == 4) {
    if (fp32_tensor_cores()) {
      gj_run_tc(descs, base, status, s, pivot_floor);
      return;
    }
  }
  gj_run<T>(descs, base, status, s, pivot_floor);
}

template <typename T>
void large_inverse(T* A, int n, int ld, int* status, cudaStream_t s, const std::vector<int32_t>* first_col) {
  if (first_col) {
    const std::vector<int> lim = gj_envelope(*first_col, n, GJWidth<T>::value);
    gj_run<T>(std::vector<InvDesc>{{n, ld, 0}}, A, status, s, T(0), &lim);
    return;
  }
  gj_run<T>(std::vector<InvDesc>{{n, ld, 0}}, A, status, s, T(0));
}

template void batched_gemm<double>(bool, bool, const std::vector<GemmDesc>&, const double*, const double*, double*,
                                   double, double, cudaStream_t);
template void batched_gemm<float>(bool, bool, const std::vector<GemmDesc>&, const float*, const float*, float*, float,
                                  float, cudaStream_t);
template void batched_inverse<double>(const std::vector<InvDesc>&, double*, int*, cudaStream_t, double);
template void batched_inverse<float>(const std::vector<InvDesc>&, float*, int*, cudaStream_t, float);
template void large_inverse<double>(double*, int, int, int*, cudaStream_t, const std::vector<int32_t>*);

}  // namespace ufe
