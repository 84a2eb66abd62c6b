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
#include <algorithm>
#include <mutex>
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
template <typename T, int NB>
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
  if (keep || I == J) return;
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

// Tiles of step K other than block row / column K+1 (one CTA per tile I <= J).
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
// tile (min(K+1, t), max(K+1, t))); the CTA of t = K+1 keeps the updated diagonal tile
// in shared memory and inverts it into Dnext, the next step's D^-1.  Grid (matrix,
// tile) with the diagonal tiles in the first grid row, so that every matrix's serial
// inversion starts in the first wave.
template <typename T, int NB>
__global__ void __launch_bounds__(kGJThreads)
k_gj_lookahead(GJBatch bt, int step, int nblk, T* __restrict__ base, const T* __restrict__ R,
               const T* __restrict__ Q, const T* __restrict__ Dg, T* __restrict__ Dnext, int* status, T floor) {
  const int b = blockIdx.x;
  const InvDesc d = bt.d[b];
  const int nd = step + 1;
  if (nd >= nblk) return;
  const int y = (int)blockIdx.y;
  const int t = y == 0 ? nd : (y <= nd ? y - 1 : y);
  const int I = min(nd, t), J = max(nd, t);
  if (step * NB >= d.n || J * NB >= d.n) return;
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

template <typename T>
static void gj_run(const std::vector<InvDesc>& descs, T* base, int* status, cudaStream_t s, T floor) {
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
  const unsigned ntri = (unsigned)(nblk * (nblk + 1) / 2);
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
      k_gj_panel<T, NB><<<dim3((nmax + pcols - 1) / pcols, nb), kGJThreads, 0, s>>>(bt, 0, pcols, base, Rc, Qc, Dc);
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
      k_gj_lookahead<T, NB><<<dim3(nb, nblk), kGJThreads, 0, s2>>>(bt, step, nblk, base, Rc, Qc, Dc, Dn, status,
                                                                   floor);
      UFE_CHECK_LAUNCH();
      ta.end(s2);
      TimedLaunch tp;
      tp.begin(sizeof(T) == 8 ? "gj_panel_f64" : "gj_panel_f32", s2);
      k_gj_panel<T, NB><<<dim3((nmax + pcols - 1) / pcols, nb), kGJThreads, 0, s2>>>(bt, step + 1, pcols, base, Rn, Qn, Dn);
      UFE_CHECK_LAUNCH();
      tp.end(s2);
    }
    TimedLaunch tl;
    tl.begin(sizeof(T) == 8 ? "gj_update_f64" : "gj_update_f32", s);
    k_gj_update<T, NB><<<dim3(ntri, nb), kGJThreads, 0, s>>>(bt, step, nblk, base, Rc, Qc, Dc);
    UFE_CHECK_LAUNCH();
    tl.end(s);
    UFE_CUDA(cudaEventRecord(ev[1], s2));
    UFE_CUDA(cudaStreamWaitEvent(s, ev[1], 0));
  }
}

template <typename T>
void batched_inverse(const std::vector<InvDesc>& descs, T* base, int* status, cudaStream_t s, T pivot_floor) {
  gj_run<T>(descs, base, status, s, pivot_floor);
}

template <typename T>
void large_inverse(T* A, int n, int ld, int* status, cudaStream_t s) {
  gj_run<T>(std::vector<InvDesc>{{n, ld, 0}}, A, status, s, T(0));
}

template void batched_gemm<double>(bool, bool, const std::vector<GemmDesc>&, const double*, const double*, double*,
                                   double, double, cudaStream_t);
template void batched_gemm<float>(bool, bool, const std::vector<GemmDesc>&, const float*, const float*, float*, float,
                                  float, cudaStream_t);
template void batched_inverse<double>(const std::vector<InvDesc>&, double*, int*, cudaStream_t, double);
template void batched_inverse<float>(const std::vector<InvDesc>&, float*, int*, cudaStream_t, float);
template void large_inverse<double>(double*, int, int, int*, cudaStream_t);

}  // namespace ufe
