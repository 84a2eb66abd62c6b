// Three-level BDDC: the coarse problem of Eq. bddc preconditioned by BDDC one level up.
//
// The paper's conclusions (Sect. 6) point to multilevel BDDC for problems whose
// coarse problem outgrows one factorisation.  The coarse problem
//   A_c = sum_w R_cw^T A_c^w R_cw   (A_c^w = Phi^wT A^w Phi^w, Sect. 3.3)
// is itself sub-assembled, with the subdomains as elements and the coarse DOFs as
// DOFs.  Level 2 builds BDDC on it the way Sect. 3 builds the first level:
//   * level-2 subdomains J: the subdomains grouped G x G x G blocks at a time, and
//     inside a group the connected components under "hold a common coarse DOF";
//   * neigh_2(k): the level-2 subdomains holding a subdomain that holds coarse DOF k;
//     the level-2 interface is {k : |neigh_2(k)| >= 2};
//   * level-2 objects: interface coarse DOFs with equal neigh_2, split into connected
//     components under "held by a common subdomain"; face when |neigh_2| = 2, else
//     corner for one coarse DOF and edge for more; the first level's choice of
//     corners / edges / faces (opts.coarse) applies;
//   * for elasticity the classes are also split by the type of first-level coarse
//     DOF (a component mean, or a rotation moment about one axis);
//   * level-2 coarse DOFs ("level 3"): the uniform mean over each object;
//   * stiffness weights from the diagonals of A_2^J = sum_{w in J} A_c^w;
//   * the level-3 matrix, assembled from Phi_2^JT A_2^J Phi_2^J, inverted exactly.
// Every level-2 operator is explicit and FP64, as at the first level: A_2,II^-1,
// the constrained Neumann operator K_2 = S'^-1 - Phi_2 X^T on the level-2 interface
// (S' = S + C^T diag(rho) C, X = S'^-1 C^T, Phi_2 = X (C X)^-1) and Phi_2 itself.
//
// One application u_c = M_2 r_c (replacing u_c = A_c^-1 r_c) is four launches:
//   L1  per J: r_c gathered from the subdomain parts; y = A_II^-1 r_I; t = A_GI y
//   L2  per J: r~ = w (r_G - sum_J' t^J'); v = K_2 r~ (stored weighted); g = Phi_2^T r~
//   L34 per J: r_3 = sum g gathered whole; u_3 on J's level-3 DOFs (rows of A_3^-1);
//       vw += w Phi_2 u_3  (a level-3 problem too large for one CTA's shared memory
//       takes two launches instead: the first level's dense coarse kernel, then the
//       prolongation)
//   L5  per J: u_G = sum_J' vw^J'; z_I = y - A_II^-1 A_IG u_G; u_c = z
#include <algorithm>
#include <cmath>
#include <deque>
#include <map>
#include <vector>

#include "bddc.cuh"
#include "dense.cuh"

namespace ufe {

namespace {

// device view of the level-2 operators (all device pointers)
struct MlMeta {
  const int32_t* dof_ptr;   // n2 + 1: local DOFs of J at dofs[dof_ptr[J] ..]: interior first, then interface
  const int32_t* nI;        // n2: interior count of J
  const int32_t* dofs;      // coarse DOF id of every local slot
  const int32_t* slot_J;    // level-2 subdomain of every local slot
  const uint8_t* owner;     // interface slot whose J is the first of neigh_2 (it writes u_c)
  const int32_t* gpos2;     // n_c x 8: local slot of coarse DOF k in the i-th level-2 subdomain of neigh_2(k)
  const uint8_t* nn2;       // n_c: |neigh_2(k)|
  const int64_t* offA;      // A_2^J (n x pad4(n)): A_II^-1 in the interior block, A_IG, A_GI, A_GG as assembled
  const int64_t* offK;      // K_2^J (nG x pad4(nG))
  const int64_t* offP;      // Phi_2^J (nG x pad4(nC))
  const int32_t* c_ptr;     // n2 + 1: level-3 DOFs of J at c_list[c_ptr[J] ..]
  const int32_t* c_list;
  const double* store;
  const double* w2;         // weight of every local slot (interface slots used)
  double* y2;               // interior slots: y = A_II^-1 r_I
  double* rc2;              // interface slots: r_c
  double* t2;               // interface slots: A_GI y
  double* vw2;              // interface slots: w K_2 r~
  double* g3;               // level-3 slots: Phi_2^T r~
  const double* u3;         // n3: level-3 solution
};

__device__ __forceinline__ double ml_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// rows [r0, r1) of a row-major block times xs[0 .. ncol): one warp per row
__device__ __forceinline__ void ml_rows(const double* __restrict__ M, int ld, int r0, int r1, int c0, int ncol,
                                        const double* __restrict__ xs, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = r0 + wid; r < r1; r += nw) {
    const double* row = M + (int64_t)r * ld + c0;
    double s = 0.0;
    for (int c = lane; c < ncol; c += 32) s += row[c] * xs[c];
    s = ml_warp_sum(s);
    if (lane == 0) out[r - r0] = s;
  }
}

// sum of v[slot[k]] over the first cnt (<= 8) of the eight slots stored for one
// coarse DOF, in slot order: the slots arrive in two 16-byte loads and the values
// are loaded together (no chain of dependent loads)
__device__ __forceinline__ double ml_gather8(const int32_t* __restrict__ slots8, int cnt,
                                             const double* __restrict__ v) {
  const int4 pa = *reinterpret_cast<const int4*>(slots8);
  const int4 pb = *reinterpret_cast<const int4*>(slots8 + 4);
  const int sl[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = k < cnt ? v[sl[k]] : 0.0;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (k < cnt) s += x[k];
  return s;
}

// L1: r_c on J's local DOFs (the subdomain parts of each coarse DOF in neighbour
// order, as the first level's dense coarse kernel sums them); y = A_II^-1 r_I; t = A_GI y
__global__ void __launch_bounds__(256)
k_ml_interior(MlMeta M, const int32_t* __restrict__ cpos, const uint8_t* __restrict__ cnn,
              const double* __restrict__ gC, const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) char smem[];
  const int J = blockIdx.x, base = M.dof_ptr[J], n = M.dof_ptr[J + 1] - base, nI = M.nI[J], ld = pad4(n);
  double* rc = reinterpret_cast<double*>(smem);
  double* y = rc + ld;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int k = M.dofs[base + i];
    const double s = ml_gather8(cpos + (int64_t)k * 8, cnn[k], gC);
    rc[i] = s;
    if (i >= nI) M.rc2[base + i] = s;
  }
  __syncthreads();
  const double* A = M.store + M.offA[J];
  ml_rows(A, ld, 0, nI, 0, nI, rc, y);
  __syncthreads();
  for (int i = threadIdx.x; i < nI; i += blockDim.x) M.y2[base + i] = y[i];
  ml_rows(A, ld, nI, n, 0, nI, y, M.t2 + base + nI);
}

// L2: r~ = w (r_G - sum over neigh_2 of A_GI y); vw = w K_2 r~; g = Phi_2^T r~ (one
// warp per column of Phi_2, lanes over its rows)
__global__ void __launch_bounds__(256) k_ml_neumann(MlMeta M, const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) char smem[];
  const int J = blockIdx.x, base = M.dof_ptr[J], n = M.dof_ptr[J + 1] - base, nI = M.nI[J], nG = n - nI;
  if (nG == 0) return;
  const int ldG = pad4(nG), c0 = M.c_ptr[J], nC = M.c_ptr[J + 1] - c0, ldC = pad4(nC);
  double* xr = reinterpret_cast<double*>(smem);
  double* v = xr + ldG;
  for (int i = threadIdx.x; i < nG; i += blockDim.x) {
    const int s0 = base + nI + i, k = M.dofs[s0];
    xr[i] = M.w2[s0] * (M.rc2[s0] - ml_gather8(M.gpos2 + (int64_t)k * 8, M.nn2[k], M.t2));
  }
  __syncthreads();
  ml_rows(M.store + M.offK[J], ldG, 0, nG, 0, nG, xr, v);
  const double* P = M.store + M.offP[J];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < nC; c += nw) {
    double s = 0.0;
    for (int i = lane; i < nG; i += 32) s += P[(int64_t)i * ldC + c] * xr[i];
    s = ml_warp_sum(s);
    if (lane == 0) M.g3[c0 + c] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nG; i += blockDim.x) M.vw2[base + nI + i] = M.w2[base + nI + i] * v[i];
}

// L4: vw += w Phi_2 u_3 on J's interface rows (u_3 of J's level-3 DOFs staged first)
__global__ void __launch_bounds__(256) k_ml_prolong(MlMeta M, const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) char smem[];
  const int J = blockIdx.x, base = M.dof_ptr[J], n = M.dof_ptr[J + 1] - base, nI = M.nI[J], nG = n - nI;
  const int c0 = M.c_ptr[J], nC = M.c_ptr[J + 1] - c0, ldC = pad4(nC);
  if (nG == 0 || nC == 0) return;
  double* u = reinterpret_cast<double*>(smem);
  double* pu = u + ldC;
  for (int c = threadIdx.x; c < nC; c += blockDim.x) u[c] = M.u3[M.c_list[c0 + c]];
  __syncthreads();
  ml_rows(M.store + M.offP[J], ldC, 0, nG, 0, nC, u, pu);
  __syncthreads();
  for (int i = threadIdx.x; i < nG; i += blockDim.x) M.vw2[base + nI + i] += M.w2[base + nI + i] * pu[i];
}

// L3 and L4 in one launch (level-3 problems whose r_3 fits shared memory): each J
// gathers the whole r_3 (the parts of every level-3 DOF from the level-2 subdomains
// holding it, in their order), forms u_3 on its own level-3 DOFs from those rows of
// A_3^-1, and adds w Phi_2 u_3 to its interface rows
__global__ void __launch_bounds__(256)
k_ml_coarse3(MlMeta M, int n3, int ld3, const double* __restrict__ A3inv, const int32_t* __restrict__ cpos3,
             const uint8_t* __restrict__ nn3, const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) char smem[];
  const int J = blockIdx.x, base = M.dof_ptr[J], n = M.dof_ptr[J + 1] - base, nI = M.nI[J], nG = n - nI;
  const int c0 = M.c_ptr[J], nC = M.c_ptr[J + 1] - c0, ldC = pad4(nC);
  if (nG == 0 || nC == 0) return;
  double* r3 = reinterpret_cast<double*>(smem);
  double* u = r3 + ld3;
  double* pu = u + ldC;
  for (int q = threadIdx.x; q < n3; q += blockDim.x) r3[q] = ml_gather8(cpos3 + (int64_t)q * 8, nn3[q], M.g3);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < nC; c += nw) {
    const double* row = A3inv + (int64_t)M.c_list[c0 + c] * ld3;
    double acc = 0.0;
    for (int j = lane; j < n3; j += 32) acc += row[j] * r3[j];
    acc = ml_warp_sum(acc);
    if (lane == 0) u[c] = acc;
  }
  __syncthreads();
  ml_rows(M.store + M.offP[J], ldC, 0, nG, 0, nC, u, pu);
  __syncthreads();
  for (int i = threadIdx.x; i < nG; i += blockDim.x) M.vw2[base + nI + i] += M.w2[base + nI + i] * pu[i];
}

// L5: u_G = sum over neigh_2 of w (K_2 r~ + Phi_2 u_3); z_I = y - A_II^-1 (A_IG u_G); u_c = z
__global__ void __launch_bounds__(256) k_ml_final(MlMeta M, double* __restrict__ uc, const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) char smem[];
  const int J = blockIdx.x, base = M.dof_ptr[J], n = M.dof_ptr[J + 1] - base, nI = M.nI[J], nG = n - nI;
  const int ld = pad4(n);
  double* ug = reinterpret_cast<double*>(smem);
  double* tI = ug + pad4(nG);
  double* zI = tI + pad4(nI);
  for (int i = threadIdx.x; i < nG; i += blockDim.x) {
    const int k = M.dofs[base + nI + i];
    const double u = ml_gather8(M.gpos2 + (int64_t)k * 8, M.nn2[k], M.vw2);
    ug[i] = u;
    if (M.owner[base + nI + i]) uc[k] = u;
  }
  __syncthreads();
  if (nI == 0) return;
  const double* A = M.store + M.offA[J];
  ml_rows(A, ld, 0, nI, nI, nG, ug, tI);
  __syncthreads();
  ml_rows(A, ld, 0, nI, 0, nI, tI, zI);
  __syncthreads();
  for (int i = threadIdx.x; i < nI; i += blockDim.x) uc[M.dofs[base + i]] = M.y2[base + i] - zI[i];
}

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------
// A_2^J = sum_{w in J} A_c^w scattered to J's local numbering (members one after
// another, so that no two threads add to one entry at once), then symmetrised (the
// A_c^w come out of inversions, symmetric only to rounding, and the inversions below
// read one triangle)
__global__ void k_ml_assemble(const int32_t* __restrict__ mem_ptr, const int32_t* __restrict__ mem_list,
                              const int32_t* __restrict__ C_ptr, const int32_t* __restrict__ loc,
                              const int64_t* __restrict__ oCC, const double* __restrict__ Acw,
                              const int32_t* __restrict__ dof_ptr, const int64_t* __restrict__ offA,
                              double* __restrict__ store) {
  const int J = blockIdx.x, n = dof_ptr[J + 1] - dof_ptr[J], ld = pad4(n);
  double* A = store + offA[J];
  for (int e = threadIdx.x; e < n * ld; e += blockDim.x) A[e] = 0.0;
  __syncthreads();
  for (int q = mem_ptr[J]; q < mem_ptr[J + 1]; ++q) {
    const int w = mem_list[q], c0 = C_ptr[w], nC = C_ptr[w + 1] - c0, ldC = pad4(nC);
    for (int e = threadIdx.x; e < nC * nC; e += blockDim.x) {
      const int i = e / nC, j = e % nC;
      A[(int64_t)loc[c0 + i] * ld + loc[c0 + j]] += Acw[oCC[w] + (int64_t)i * ldC + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    if (j <= i) continue;
    const double v = 0.5 * (A[(int64_t)i * ld + j] + A[(int64_t)j * ld + i]);
    A[(int64_t)i * ld + j] = v;
    A[(int64_t)j * ld + i] = v;
  }
}

// symmetric Jacobi scaling around an in-place inversion: pass 0 computes s = diag^-1/2
// (DEV_SINGULAR for a non-positive diagonal) and scales, pass 1 scales the inverse
// again (inv(A) = S inv(S A S) S)
__global__ void k_ml_jacobi(const InvDesc* __restrict__ d, const int64_t* __restrict__ soff, double* __restrict__ sv,
                            double* __restrict__ store, int pass, int* __restrict__ status) {
  const InvDesc D = d[blockIdx.x];
  double* A = store + D.off;
  double* s = sv + soff[blockIdx.x];
  if (pass == 0) {
    for (int i = threadIdx.x; i < D.n; i += blockDim.x) {
      const double a = A[(int64_t)i * D.ld + i];
      if (!(a > 0.0)) atomicOr(status + blockIdx.x, DEV_SINGULAR);
      s[i] = a > 0.0 ? 1.0 / sqrt(a) : 1.0;
    }
    __syncthreads();
  }
  for (int64_t e = threadIdx.x; e < (int64_t)D.n * D.n; e += blockDim.x) {
    const int i = (int)(e / D.n), j = (int)(e % D.n);
    A[(int64_t)i * D.ld + j] *= s[i] * s[j];
  }
}

// S = A_GG (copied out of A_2)
__global__ void k_ml_copy_gg(const int32_t* __restrict__ dof_ptr, const int32_t* __restrict__ nIv,
                             const int64_t* __restrict__ offA, const int64_t* __restrict__ offK,
                             double* __restrict__ store) {
  const int J = blockIdx.x, n = dof_ptr[J + 1] - dof_ptr[J], nI = nIv[J], nG = n - nI, ld = pad4(n), ldG = pad4(nG);
  const double* A = store + offA[J];
  double* S = store + offK[J];
  for (int e = threadIdx.x; e < nG * nG; e += blockDim.x) {
    const int i = e / nG, j = e % nG;
    S[(int64_t)i * ldG + j] = A[(int64_t)(nI + i) * ld + nI + j];
  }
}

// Jacobi scaling of the level-2 problem of J (as at the first level): s = diag(A_2)^-1/2
// over J's local DOFs, A^ = S A S, constraint rows C^ = C S_G with rho_q = 1 / |C^_q|^2
// (each row summed in order by one thread); DEV_SINGULAR for a non-positive diagonal
__global__ void k_ml_scale(const int32_t* __restrict__ dof_ptr, const int32_t* __restrict__ nIv,
                           const int32_t* __restrict__ c_ptr, const int64_t* __restrict__ offA,
                           const int64_t* __restrict__ offC, double* __restrict__ sv, double* __restrict__ rho,
                           double* __restrict__ store, int* __restrict__ status) {
  const int J = blockIdx.x, base = dof_ptr[J], n = dof_ptr[J + 1] - base, nI = nIv[J], nG = n - nI;
  const int ld = pad4(n), ldG = pad4(nG), c0 = c_ptr[J], nC = c_ptr[J + 1] - c0;
  double* A = store + offA[J];
  double* C = store + offC[J];
  double* sj = sv + base;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = A[(int64_t)i * ld + i];
    if (!(a > 0.0)) atomicOr(status, DEV_SINGULAR);
    sj[i] = a > 0.0 ? 1.0 / sqrt(a) : 1.0;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    A[(int64_t)i * ld + j] *= sj[i] * sj[j];
  }
  for (int e = threadIdx.x; e < nC * nG; e += blockDim.x) {
    const int q = e / nG, i = e % nG;
    C[(int64_t)q * ldG + i] *= sj[nI + i];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nC; q += blockDim.x) {
    double nrm = 0.0;
    for (int i = 0; i < nG; ++i) nrm += C[(int64_t)q * ldG + i] * C[(int64_t)q * ldG + i];
    rho[c0 + q] = nrm > 0.0 ? 1.0 / nrm : 0.0;
  }
}

// back to the unscaled variables for the iterations: A_II^-1 = S P^ S, the assembled
// off-diagonal blocks A = S^-1 A^ S^-1, K_2 = S_G K^ S_G, Phi_2 = S_G Phi^
__global__ void k_ml_unscale(const int32_t* __restrict__ dof_ptr, const int32_t* __restrict__ nIv,
                             const int32_t* __restrict__ c_ptr, const int64_t* __restrict__ offA,
                             const int64_t* __restrict__ offK, const int64_t* __restrict__ offP,
                             const double* __restrict__ sv, double* __restrict__ store) {
  const int J = blockIdx.x, base = dof_ptr[J], n = dof_ptr[J + 1] - base, nI = nIv[J], nG = n - nI;
  const int ld = pad4(n), ldG = pad4(nG), nC = c_ptr[J + 1] - c_ptr[J], ldC = pad4(nC);
  const double* sj = sv + base;
  double* A = store + offA[J];
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i < nI && j < nI)
      A[(int64_t)i * ld + j] *= sj[i] * sj[j];
    else
      A[(int64_t)i * ld + j] /= sj[i] * sj[j];
  }
  double* K = store + offK[J];
  for (int e = threadIdx.x; e < nG * nG; e += blockDim.x) {
    const int i = e / nG, j = e % nG;
    K[(int64_t)i * ldG + j] *= sj[nI + i] * sj[nI + j];
  }
  double* P = store + offP[J];
  for (int e = threadIdx.x; e < nG * nC; e += blockDim.x) {
    const int i = e / nC, c = e % nC;
    P[(int64_t)i * ldC + c] *= sj[nI + i];
  }
}

// S' = sym(S) + C^T diag(rho) C (scaled variables)
__global__ void k_ml_penalty(const int32_t* __restrict__ dof_ptr, const int32_t* __restrict__ nIv,
                             const int32_t* __restrict__ c_ptr, const int64_t* __restrict__ offK,
                             const int64_t* __restrict__ offC, const double* __restrict__ rho,
                             double* __restrict__ store) {
  const int J = blockIdx.x, nG = dof_ptr[J + 1] - dof_ptr[J] - nIv[J], ldG = pad4(nG);
  const int c0 = c_ptr[J], nC = c_ptr[J + 1] - c0;
  double* S = store + offK[J];
  const double* C = store + offC[J];
  for (int e = threadIdx.x; e < nG * nG; e += blockDim.x) {
    const int i = e / nG, j = e % nG;
    if (j < i) continue;
    double pen = 0.0;
    for (int q = 0; q < nC; ++q) pen += rho[c0 + q] * C[(int64_t)q * ldG + i] * C[(int64_t)q * ldG + j];
    const double v = 0.5 * (S[(int64_t)i * ldG + j] + S[(int64_t)j * ldG + i]) + pen;
    S[(int64_t)i * ldG + j] = v;
    S[(int64_t)j * ldG + i] = v;
  }
}

// A_3^J = (C S'^-1 C^T)^-1 - diag(rho), symmetrised
__global__ void k_ml_coarse_local(const int32_t* __restrict__ c_ptr, const int64_t* __restrict__ offSc,
                                  const double* __restrict__ rho, double* __restrict__ store) {
  const int J = blockIdx.x, c0 = c_ptr[J], nC = c_ptr[J + 1] - c0, ldC = pad4(nC);
  double* A = store + offSc[J];
  for (int e = threadIdx.x; e < nC * nC; e += blockDim.x) {
    const int i = e / nC, j = e % nC;
    if (j < i) continue;
    double v = 0.5 * (A[(int64_t)i * ldC + j] + A[(int64_t)j * ldC + i]);
    if (i == j) v -= rho[c0 + i];
    A[(int64_t)i * ldC + j] = v;
    A[(int64_t)j * ldC + i] = v;
  }
}

// level-3 matrix: row q gathers A_3^J of every level-2 subdomain holding it, in order
__global__ void k_ml_a3_assemble(int n3, int ld3, const int32_t* __restrict__ cpos3, const uint8_t* __restrict__ nn3,
                                 const int32_t* __restrict__ slot_J3, const int32_t* __restrict__ c_ptr,
                                 const int32_t* __restrict__ c_list, const int64_t* __restrict__ offSc,
                                 const double* __restrict__ store, double* __restrict__ A3) {
  const int q = blockIdx.x;
  for (int j = threadIdx.x; j < ld3; j += blockDim.x) A3[(int64_t)q * ld3 + j] = 0.0;
  __syncthreads();
  for (int h = 0; h < nn3[q]; ++h) {
    const int sl = cpos3[(int64_t)q * 8 + h], J = slot_J3[sl];
    const int c0 = c_ptr[J], nC = c_ptr[J + 1] - c0, ldC = pad4(nC), r = sl - c0;
    const double* row = store + offSc[J] + (int64_t)r * ldC;
    for (int j = threadIdx.x; j < nC; j += blockDim.x) A3[(int64_t)q * ld3 + c_list[c0 + j]] += row[j];
    __syncthreads();
  }
}

// stiffness weights of the interface slots: A_2^J_kk / sum over neigh_2(k) (the diagonal
// of the A_GG block, which the interior inversion leaves as assembled); 1 elsewhere
__global__ void k_ml_diag(int64_t n_slots, const int32_t* __restrict__ slot_J, const int32_t* __restrict__ dof_ptr,
                          const int32_t* __restrict__ nIv, const int64_t* __restrict__ offA,
                          const double* __restrict__ store, double* __restrict__ d2) {
  const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= n_slots) return;
  const int J = slot_J[sl], i = (int)(sl - dof_ptr[J]), ld = pad4(dof_ptr[J + 1] - dof_ptr[J]);
  d2[sl] = i >= nIv[J] ? store[offA[J] + (int64_t)i * ld + i] : 0.0;
}
__global__ void k_ml_weights(int64_t n_slots, const int32_t* __restrict__ slot_J, const int32_t* __restrict__ dof_ptr,
                             const int32_t* __restrict__ nIv, const int32_t* __restrict__ dofs,
                             const int32_t* __restrict__ gpos2, const uint8_t* __restrict__ nn2,
                             const double* __restrict__ d2, int topological, double* __restrict__ w2) {
  const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= n_slots) return;
  const int J = slot_J[sl], i = (int)(sl - dof_ptr[J]);
  if (i < nIv[J]) {
    w2[sl] = 1.0;
    return;
  }
  const int k = dofs[sl], cnt = nn2[k];
  if (topological) {
    w2[sl] = 1.0 / cnt;
    return;
  }
  double tot = 0.0;
  for (int j = 0; j < cnt; ++j) tot += d2[gpos2[(int64_t)k * 8 + j]];
  w2[sl] = d2[sl] / tot;
}

template <typename T>
void upload_vec(DBuf<T>& d, const std::vector<T>& v, cudaStream_t s) {
  d.alloc(std::max<size_t>(v.size(), 1), s);
  if (!v.empty()) UFE_CUDA(cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

MlMeta meta_of(const MultiLevel& L) {
  MlMeta M;
  M.dof_ptr = L.dof_ptr.p;
  M.nI = L.nI.p;
  M.dofs = L.dofs.p;
  M.slot_J = L.slot_J.p;
  M.owner = L.owner.p;
  M.gpos2 = L.gpos2.p;
  M.nn2 = L.nn2.p;
  M.offA = L.offA.p;
  M.offK = L.offK.p;
  M.offP = L.offP.p;
  M.c_ptr = L.c_ptr.p;
  M.c_list = L.c_list.p;
  M.store = L.store.p;
  M.w2 = L.w2.p;
  M.y2 = L.y2.p;
  M.rc2 = L.rc2.p;
  M.t2 = L.t2.p;
  M.vw2 = L.vw2.p;
  M.g3 = L.g3.p;
  M.u3 = L.u3.p;
  return M;
}

// the scaled in-place inversion of a batch of SPD blocks of the arena
// the status flags of every inversion, read once at the end of the set-up
struct StatusList {
  std::deque<DBuf<int>> bufs;
  int* next(size_t n, cudaStream_t s) {
    bufs.emplace_back();
    bufs.back().alloc(n, s);
    bufs.back().zero();
    return bufs.back().p;
  }
  bool any(cudaStream_t s) const {
    std::vector<std::vector<int>> h;
    for (const DBuf<int>& b : bufs) {
      h.emplace_back(b.n);
      UFE_CUDA(cudaMemcpyAsync(h.back().data(), b.p, b.n * sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    UFE_CUDA(cudaStreamSynchronize(s));
    for (const auto& v : h)
      for (int x : v)
        if (x & (DEV_SINGULAR | DEV_ILLCOND)) return true;
    return false;
  }
};

void scaled_inverse(const std::vector<InvDesc>& descs, double* store, StatusList& sl, cudaStream_t s) {
  std::vector<InvDesc> d;
  std::vector<int64_t> so;
  int64_t ns = 0;
  for (const InvDesc& x : descs)
    if (x.n > 0) {
      d.push_back(x);
      so.push_back(ns);
      ns += x.n;
    }
  if (d.empty()) return;
  DBuf<InvDesc> dd;
  DBuf<int64_t> ds;
  DBuf<double> sv;
  upload_vec(dd, d, s);
  upload_vec(ds, so, s);
  sv.alloc(ns, s);
  int* st = sl.next(d.size(), s);
  k_ml_jacobi<<<(unsigned)d.size(), 256, 0, s>>>(dd.p, ds.p, sv.p, store, 0, st);
  UFE_CHECK_LAUNCH();
  // unit diagonals after the scaling: a pivot at rounding level means a singular block
  // (a level-2 subdomain that floats without a level-2 coarse DOF)
  batched_inverse<double>(d, store, st, s, 1e-15);
  k_ml_jacobi<<<(unsigned)d.size(), 256, 0, s>>>(dd.p, ds.p, sv.p, store, 1, st);
  UFE_CHECK_LAUNCH();
  // the buffers above are released stream-ordered, after the kernels that read them
}

}  // namespace

// level-3 problems up to this many bytes of r_3 (plus J's vectors) take the fused launch
constexpr size_t kFusedCoarse3Smem = 160 * 1024;

void ml_prepare(int max_n, int max_nI, int max_nG, int max_nC, int ld3);

void ml_setup(Bddc& B, const DBuf<double>& Acw, const std::vector<int64_t>& hCC, int group, cudaStream_t s) {
  MultiLevel& L = B.ml;
  const Mesh& m = *B.mesh;
  const int ns = (int)m.n_sub;
  const int64_t nc = B.n_coarse;
  UFE_REQUIRE(group >= 1, UFE_ERR_INVALID_ARG, "coarse_group must be positive");
  L.n2 = 0;
  if (nc == 0) return;
  // ---- host bookkeeping of the level-2 partition (integer work on the subdomain graph)
  const std::vector<int32_t> Cp = to_host(B.C_ptr.p, ns + 1, s);
  const std::vector<int32_t> Cl = to_host(B.C_list.p, Cp[ns], s);
  const std::vector<int32_t> blk = to_host(m.sub_block.p, ns, s);
  std::vector<std::vector<int>> holders(nc);
  for (int w = 0; w < ns; ++w)
    for (int c = Cp[w]; c < Cp[w + 1]; ++c) holders[Cl[c]].push_back(w);
  const GridGeom& g = m.g;
  const int gx = (g.bx + group - 1) / group, gy = (g.by + group - 1) / group;
  std::vector<int> grp(ns);
  for (int w = 0; w < ns; ++w) {
    const int b = blk[w], bi = b % g.bx, bj = (b / g.bx) % g.by, bk = b / (g.bx * g.by);
    grp[w] = bi / group + gx * (bj / group + gy * (bk / group));
  }
  std::vector<int> J_of(ns, -1);
  std::vector<std::vector<int>> members;
  for (int w0 = 0; w0 < ns; ++w0) {
    if (J_of[w0] >= 0) continue;
    const int J = (int)members.size();
    std::vector<int> comp{w0};
    J_of[w0] = J;
    std::deque<int> queue{w0};
    while (!queue.empty()) {
      const int w = queue.front();
      queue.pop_front();
      for (int c = Cp[w]; c < Cp[w + 1]; ++c)
        for (int w2 : holders[Cl[c]])
          if (J_of[w2] < 0 && grp[w2] == grp[w0]) {
            J_of[w2] = J;
            comp.push_back(w2);
            queue.push_back(w2);
          }
    }
    std::sort(comp.begin(), comp.end());
    members.push_back(comp);
  }
  const int n2 = (int)members.size();
  std::vector<std::vector<int>> neigh2(nc);
  for (int64_t k = 0; k < nc; ++k) {
    for (int w : holders[k]) neigh2[k].push_back(J_of[w]);
    std::sort(neigh2[k].begin(), neigh2[k].end());
    neigh2[k].erase(std::unique(neigh2[k].begin(), neigh2[k].end()), neigh2[k].end());
    UFE_REQUIRE(neigh2[k].size() <= 8, UFE_ERR_INVALID_ARG, "a coarse DOF held by more than 8 level-2 subdomains");
  }
  // level-2 objects: classes of equal neigh_2 split into components under "held by a
  // common subdomain", ordered by smallest coarse DOF
  struct Obj {
    std::vector<int> dofs, neigh;
    int kind;
  };
  std::vector<Obj> objs;
  {
    // the type of each first-level coarse DOF: its row within the object's rows, the
    // component means first (0 .. ncomp-1), then the rotation moments about the kept
    // axes k in increasing order (3 + k); classes are split by type, so that a level-2
    // coarse DOF averages one kind of first-level coarse DOF
    const std::vector<int32_t> cobj = to_host(B.coarse_obj.p, nc, s);
    const std::vector<int32_t> cfirst = to_host(B.coarse_of_obj.p, B.n_obj, s);
    const std::vector<int32_t> orot = to_host(B.obj_rot.p, B.n_obj, s);
    std::vector<int32_t> type1(nc);
    for (int64_t k = 0; k < nc; ++k) {
      const int o = cobj[k], r = (int)(k - cfirst[o]);
      int t = r;
      if (r >= B.ncomp) {
        for (int axis = 0, seen = 0; axis < 3; ++axis)
          if ((orot[o] >> axis) & 1) {
            if (seen == r - B.ncomp) t = 3 + axis;
            ++seen;
          }
      }
      type1[k] = t;
    }
    // with coarse_keep_corners, a coarse DOF of a first-level corner is a level-2 corner
    std::vector<int32_t> kind1;
    if (B.coarse_keep_corners) {
      const std::vector<int32_t> okind = to_host(B.obj_kind.p, B.n_obj, s);
      kind1.resize(nc);
      for (int64_t k = 0; k < nc; ++k) kind1[k] = okind[cobj[k]];
    }
    // key: the type, then neigh_2
    std::map<std::vector<int>, std::vector<int>> classes;
    for (int64_t k = 0; k < nc; ++k)
      if (neigh2[k].size() >= 2) {
        if (!kind1.empty() && kind1[k] == UFE_OBJ_CORNER) {
          objs.push_back(Obj{{(int)k}, neigh2[k], UFE_OBJ_CORNER});
        } else {
          std::vector<int> key{type1[k]};
          key.insert(key.end(), neigh2[k].begin(), neigh2[k].end());
          classes[key].push_back((int)k);
        }
      }
    std::vector<int> cls(nc, -1), seen(nc, 0);
    int ci = 0;
    for (auto& kv : classes) {
      for (int k : kv.second) cls[k] = ci;
      for (int k0 : kv.second) {
        if (seen[k0]) continue;
        std::vector<int> comp{k0};
        seen[k0] = 1;
        std::deque<int> queue{k0};
        while (!queue.empty()) {
          const int k = queue.front();
          queue.pop_front();
          for (int w : holders[k])
            for (int c = Cp[w]; c < Cp[w + 1]; ++c) {
              const int k2 = Cl[c];
              if (cls[k2] == ci && !seen[k2]) {
                seen[k2] = 1;
                comp.push_back(k2);
                queue.push_back(k2);
              }
            }
        }
        std::sort(comp.begin(), comp.end());
        const std::vector<int> ns2(kv.first.begin() + 1, kv.first.end());
        const int kind = ns2.size() == 2 ? UFE_OBJ_FACE : (comp.size() == 1 ? UFE_OBJ_CORNER : UFE_OBJ_EDGE);
        const bool keep = kind == UFE_OBJ_CORNER || (kind == UFE_OBJ_EDGE && B.opts.coarse != UFE_COARSE_C) ||
                          (kind == UFE_OBJ_FACE && B.opts.coarse == UFE_COARSE_CEF);
        if (keep) objs.push_back(Obj{comp, ns2, kind});
      }
      ++ci;
    }
    std::sort(objs.begin(), objs.end(), [](const Obj& a, const Obj& b) { return a.dofs[0] < b.dofs[0]; });
  }
  const int n3 = (int)objs.size();
  // local numbering of each J: interior coarse DOFs then interface ones, each ascending
  std::vector<int32_t> dof_ptr(n2 + 1, 0), nI(n2), dofs, slot_J, c_ptr(n2 + 1, 0), c_list, mem_ptr(n2 + 1, 0),
      mem_list, loc(Cp[ns]), gpos2(nc * 8, -1), cpos3((int64_t)n3 * 8, -1), slot_J3;
  std::vector<uint8_t> owner, nn2(nc), nn3(n3);
  std::vector<std::vector<int>> oids(n2);
  for (int q = 0; q < n3; ++q) {
    nn3[q] = (uint8_t)objs[q].neigh.size();
    for (int J : objs[q].neigh) oids[J].push_back(q);
  }
  std::vector<int64_t> offA(n2), offK(n2), offC(n2), offX(n2), offSc(n2), offP(n2), offT(n2);
  int64_t arena = 0;
  auto take = [&](int64_t count) {
    const int64_t o = arena;
    arena += (count + 3) & ~int64_t(3);
    return o;
  };
  std::vector<int> pos_of(nc, -1);
  int max_n = 0, max_nI = 0, max_nG = 0;
  std::vector<std::pair<int64_t, std::vector<double>>> cblocks;
  for (int J = 0; J < n2; ++J) {
    std::vector<int> loc_dofs;
    for (int w : members[J]) {
      mem_list.push_back(w);
      for (int c = Cp[w]; c < Cp[w + 1]; ++c) loc_dofs.push_back(Cl[c]);
    }
    mem_ptr[J + 1] = (int32_t)mem_list.size();
    std::sort(loc_dofs.begin(), loc_dofs.end());
    loc_dofs.erase(std::unique(loc_dofs.begin(), loc_dofs.end()), loc_dofs.end());
    std::vector<int> Ii, Gi;
    for (int k : loc_dofs) (neigh2[k].size() >= 2 ? Gi : Ii).push_back(k);
    const int n = (int)loc_dofs.size(), nIJ = (int)Ii.size(), nGJ = (int)Gi.size(), nCJ = (int)oids[J].size();
    nI[J] = nIJ;
    max_n = std::max(max_n, n);
    max_nI = std::max(max_nI, nIJ);
    max_nG = std::max(max_nG, nGJ);
    const int base = (int)dofs.size();
    for (int k : Ii) dofs.push_back(k);
    for (int k : Gi) dofs.push_back(k);
    for (int i = 0; i < n; ++i) {
      const int k = dofs[base + i];
      pos_of[k] = i;
      slot_J.push_back(J);
      owner.push_back(i >= nIJ && neigh2[k][0] == J);
      if (i >= nIJ) {
        const int h = (int)(std::find(neigh2[k].begin(), neigh2[k].end(), J) - neigh2[k].begin());
        gpos2[(int64_t)k * 8 + h] = base + i;
      }
    }
    dof_ptr[J + 1] = (int32_t)dofs.size();
    for (int w : members[J])
      for (int c = Cp[w]; c < Cp[w + 1]; ++c) loc[c] = pos_of[Cl[c]];
    for (int r = 0; r < nCJ; ++r) {
      const int q = oids[J][r];
      c_list.push_back(q);
      slot_J3.push_back(J);
      const int h = (int)(std::find(objs[q].neigh.begin(), objs[q].neigh.end(), J) - objs[q].neigh.begin());
      cpos3[(int64_t)q * 8 + h] = c_ptr[J] + r;
    }
    c_ptr[J + 1] = (int32_t)c_list.size();
    const int ld = pad4(n), ldG = pad4(nGJ), ldC = pad4(nCJ);
    offA[J] = take((int64_t)n * ld);
    offK[J] = take((int64_t)nGJ * ldG);
    offC[J] = take((int64_t)nCJ * ldG);
    offX[J] = take((int64_t)nGJ * ldC);
    offSc[J] = take((int64_t)nCJ * ldC);
    offP[J] = take((int64_t)nGJ * ldC);
    offT[J] = take((int64_t)nIJ * ldG);
    std::vector<double> cm((size_t)nCJ * ldG, 0.0);
    for (int r = 0; r < nCJ; ++r) {
      const Obj& o = objs[oids[J][r]];
      for (int k : o.dofs) cm[(size_t)r * ldG + (pos_of[k] - nIJ)] = 1.0 / (double)o.dofs.size();
    }
    cblocks.emplace_back(offC[J], std::move(cm));
  }
  for (int64_t k = 0; k < nc; ++k) nn2[k] = (uint8_t)(neigh2[k].size() >= 2 ? neigh2[k].size() : 0);
  UFE_REQUIRE(max_n <= 6144, UFE_ERR_UNSUPPORTED, "a level-2 subdomain holds more than 6144 coarse DOFs");

  // ---- device data
  L.n2 = n2;
  L.n3 = n3;
  L.ld3 = pad4(std::max(n3, 1));
  L.n_slots = (int64_t)dofs.size();
  L.max_n = max_n;
  L.max_nI = max_nI;
  L.max_nG = max_nG;
  L.max_nC = 0;
  for (int J = 0; J < n2; ++J) L.max_nC = std::max(L.max_nC, c_ptr[J + 1] - c_ptr[J]);
  L.n_obj2 = n3;
  upload_vec(L.dof_ptr, dof_ptr, s);
  upload_vec(L.nI, nI, s);
  upload_vec(L.dofs, dofs, s);
  upload_vec(L.slot_J, slot_J, s);
  upload_vec(L.owner, owner, s);
  upload_vec(L.gpos2, gpos2, s);
  upload_vec(L.nn2, nn2, s);
  upload_vec(L.offA, offA, s);
  upload_vec(L.offP, offP, s);
  upload_vec(L.c_ptr, c_ptr, s);
  upload_vec(L.c_list, c_list, s);
  upload_vec(L.cpos3, cpos3, s);
  upload_vec(L.nn3, nn3, s);
  L.store.alloc(std::max<int64_t>(arena, 4), s);
  for (auto& cb : cblocks)
    if (!cb.second.empty())
      UFE_CUDA(cudaMemcpyAsync(L.store.p + cb.first, cb.second.data(), cb.second.size() * 8, cudaMemcpyHostToDevice,
                               s));
  DBuf<int32_t> dmem_ptr, dmem_list, dloc, dslot_J3;
  DBuf<int64_t> dCC, doffC, doffSc;
  upload_vec(dmem_ptr, mem_ptr, s);
  upload_vec(dmem_list, mem_list, s);
  upload_vec(dloc, loc, s);
  upload_vec(dslot_J3, slot_J3, s);
  upload_vec(dCC, hCC, s);
  upload_vec(doffC, offC, s);
  upload_vec(doffSc, offSc, s);
  upload_vec(L.offK, offK, s);

  // ---- level-2 operators
  k_ml_assemble<<<n2, 256, 0, s>>>(dmem_ptr.p, dmem_list.p, B.C_ptr.p, dloc.p, dCC.p, Acw.p, L.dof_ptr.p, L.offA.p,
                                   L.store.p);
  UFE_CHECK_LAUNCH();
  L.w2.alloc(std::max<int64_t>(L.n_slots, 1), s);
  {
    DBuf<double> d2;
    d2.alloc(std::max<int64_t>(L.n_slots, 1), s);
    k_ml_diag<<<grid_for(L.n_slots, 256), 256, 0, s>>>(L.n_slots, L.slot_J.p, L.dof_ptr.p, L.nI.p, L.offA.p,
                                                       L.store.p, d2.p);
    UFE_CHECK_LAUNCH();
    k_ml_weights<<<grid_for(L.n_slots, 256), 256, 0, s>>>(L.n_slots, L.slot_J.p, L.dof_ptr.p, L.nI.p, L.dofs.p,
                                                          L.gpos2.p, L.nn2.p, d2.p,
                                                          B.opts.weighting == UFE_WEIGHT_TOPOLOGICAL, L.w2.p);
    UFE_CHECK_LAUNCH();
  }
  std::vector<InvDesc> dII, dS, dSc;
  std::vector<GemmDesc> gT, gS, gX, gSc, gP, gK;
  double flops = 0.0;
  for (int J = 0; J < n2; ++J) {
    const int n = dof_ptr[J + 1] - dof_ptr[J], nIJ = nI[J], nGJ = n - nIJ, nCJ = c_ptr[J + 1] - c_ptr[J];
    const int ld = pad4(n), ldG = pad4(nGJ), ldC = pad4(nCJ);
    dII.push_back(InvDesc{nIJ, ld, offA[J]});
    dS.push_back(InvDesc{nGJ, ldG, offK[J]});
    dSc.push_back(InvDesc{nCJ, ldC, offSc[J]});
    flops += std::pow((double)nIJ, 3) + std::pow((double)nGJ, 3) + std::pow((double)nCJ, 3);
    // T = A_II^-1 A_IG;  S = A_GG - A_GI T
    gT.push_back(GemmDesc{nIJ, nGJ, nIJ, ld, ld, ldG, offA[J], offA[J] + nIJ, offT[J]});
    gS.push_back(GemmDesc{nGJ, nGJ, nIJ, ld, ldG, ldG, offA[J] + (int64_t)nIJ * ld, offT[J], offK[J]});
    // X = S'^-1 C^T;  Sc = C X;  Phi = X Sc^-1;  K = S'^-1 - Phi X^T
    gX.push_back(GemmDesc{nGJ, nCJ, nGJ, ldG, ldG, ldC, offK[J], offC[J], offX[J]});
    gSc.push_back(GemmDesc{nCJ, nCJ, nGJ, ldG, ldC, ldC, offC[J], offX[J], offSc[J]});
    gP.push_back(GemmDesc{nGJ, nCJ, nCJ, ldC, ldC, ldC, offX[J], offSc[J], offP[J]});
    gK.push_back(GemmDesc{nGJ, nGJ, nCJ, ldC, ldC, ldG, offP[J], offX[J], offK[J]});
  }
  double* st = L.store.p;
  DBuf<double> rho, sv;
  rho.alloc(std::max<int64_t>((int64_t)c_list.size(), 1), s);
  sv.alloc(std::max<int64_t>(L.n_slots, 1), s);
  StatusList status;
  k_ml_scale<<<n2, 256, 0, s>>>(L.dof_ptr.p, L.nI.p, L.c_ptr.p, L.offA.p, doffC.p, sv.p, rho.p, st,
                                status.next(1, s));
  UFE_CHECK_LAUNCH();
  scaled_inverse(dII, st, status, s);
  k_ml_copy_gg<<<n2, 256, 0, s>>>(L.dof_ptr.p, L.nI.p, L.offA.p, L.offK.p, st);
  UFE_CHECK_LAUNCH();
  batched_gemm<double>(false, false, gT, st, st, st, 1.0, 0.0, s);
  batched_gemm<double>(false, false, gS, st, st, st, -1.0, 1.0, s);
  k_ml_penalty<<<n2, 256, 0, s>>>(L.dof_ptr.p, L.nI.p, L.c_ptr.p, L.offK.p, doffC.p, rho.p, st);
  UFE_CHECK_LAUNCH();
  scaled_inverse(dS, st, status, s);
  batched_gemm<double>(false, true, gX, st, st, st, 1.0, 0.0, s);
  batched_gemm<double>(false, false, gSc, st, st, st, 1.0, 0.0, s);
  scaled_inverse(dSc, st, status, s);
  batched_gemm<double>(false, false, gP, st, st, st, 1.0, 0.0, s);
  batched_gemm<double>(false, true, gK, st, st, st, -1.0, 1.0, s);
  k_ml_coarse_local<<<n2, 256, 0, s>>>(L.c_ptr.p, doffSc.p, rho.p, st);
  UFE_CHECK_LAUNCH();
  k_ml_unscale<<<n2, 256, 0, s>>>(L.dof_ptr.p, L.nI.p, L.c_ptr.p, L.offA.p, L.offK.p, L.offP.p, sv.p, st);
  UFE_CHECK_LAUNCH();
  // ---- level 3: assembled and inverted (scaled) in FP64
  if (n3 > 0) {
    L.A3inv.alloc((int64_t)n3 * L.ld3, s);
    k_ml_a3_assemble<<<n3, 128, 0, s>>>(n3, L.ld3, L.cpos3.p, L.nn3.p, dslot_J3.p, L.c_ptr.p, L.c_list.p, doffSc.p,
                                        st, L.A3inv.p);
    UFE_CHECK_LAUNCH();
    DBuf<InvDesc> dd;
    DBuf<int64_t> ds;
    DBuf<double> sv3;
    upload_vec(dd, std::vector<InvDesc>{InvDesc{n3, L.ld3, 0}}, s);
    upload_vec(ds, std::vector<int64_t>{0}, s);
    sv3.alloc(n3, s);
    int* st3 = status.next(1, s);
    k_ml_jacobi<<<1, 256, 0, s>>>(dd.p, ds.p, sv3.p, L.A3inv.p, 0, st3);
    UFE_CHECK_LAUNCH();
    // level-3 DOFs q and q' couple only through a level-2 subdomain holding both, so
    // row q's first nonzero is the smallest level-3 DOF of any of its holders: the
    // inversion skips the blocks outside that envelope (objects follow the grid)
    std::vector<int32_t> first_col(n3);
    for (int q = 0; q < n3; ++q) {
      int f = q;
      for (int J : objs[q].neigh) f = std::min(f, oids[J].front());
      first_col[q] = f;
    }
    large_inverse<double>(L.A3inv.p, n3, L.ld3, st3, s, &first_col);
    k_ml_jacobi<<<1, 256, 0, s>>>(dd.p, ds.p, sv3.p, L.A3inv.p, 1, st3);
    UFE_CHECK_LAUNCH();
    flops += std::pow((double)n3, 3);
  }
  UFE_REQUIRE(!status.any(s), UFE_ERR_SINGULAR_COARSE,
              "a level-2 or level-3 matrix of the three-level coarse solver is not positive definite");
  // ---- per-iteration work space
  L.y2.alloc(std::max<int64_t>(L.n_slots, 1), s);
  L.rc2.alloc(std::max<int64_t>(L.n_slots, 1), s);
  L.t2.alloc(std::max<int64_t>(L.n_slots, 1), s);
  L.vw2.alloc(std::max<int64_t>(L.n_slots, 1), s);
  L.g3.alloc(std::max<int64_t>((int64_t)c_list.size(), 1), s);
  L.u3.alloc(std::max<int64_t>(n3, 1), s);
  L.u3.zero();
  // bytes one application reads: A_2 twice (interior block) and once (the rest), K_2,
  // Phi_2 (twice), the level-3 inverse
  double bytes = 0.0;
  for (int J = 0; J < n2; ++J) {
    const double n = dof_ptr[J + 1] - dof_ptr[J], nIJ = nI[J], nGJ = n - nIJ, nCJ = c_ptr[J + 1] - c_ptr[J];
    bytes += 8.0 * (2 * nIJ * nIJ + 2 * nGJ * nIJ + nGJ * nGJ + 2 * nGJ * nCJ);
  }
  L.bytes = bytes + 8.0 * n3 * (double)L.ld3;
  L.inv_flops = flops;
  ml_prepare(L.max_n, L.max_nI, L.max_nG, L.max_nC, L.ld3);
  if (n3 > 0) dense_coarse_prepare(n3, L.ld3);
  // the host tables the uploads above read go out of scope here
  UFE_CUDA(cudaStreamSynchronize(s));
}

void ml_prepare(int max_n, int max_nI, int max_nG, int max_nC, int ld3) {
  const size_t s34 = (size_t)(ld3 + pad4(max_nC) + pad4(max_nG)) * 8;
  if (s34 <= kFusedCoarse3Smem) {
    if (s34 > 48 * 1024)
      UFE_CUDA(cudaFuncSetAttribute(k_ml_coarse3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s34));
    cudaFuncAttributes fa3;
    UFE_CUDA(cudaFuncGetAttributes(&fa3, k_ml_coarse3));
  }
  const size_t a = (size_t)(pad4(max_n) + pad4(max_nI)) * 8, b = (size_t)2 * pad4(max_nG) * 8,
               c = (size_t)(pad4(max_nG) + 2 * pad4(max_nI)) * 8, d = (size_t)(pad4(max_nC) + pad4(max_nG)) * 8;
  const size_t need = std::max(std::max(a, d), std::max(b, c));
  if (need > 48 * 1024) {
    UFE_CUDA(cudaFuncSetAttribute(k_ml_interior, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
    UFE_CUDA(cudaFuncSetAttribute(k_ml_neumann, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
    UFE_CUDA(cudaFuncSetAttribute(k_ml_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
    UFE_CUDA(cudaFuncSetAttribute(k_ml_prolong, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
  } else {
    cudaFuncAttributes fa;
    UFE_CUDA(cudaFuncGetAttributes(&fa, k_ml_interior));
    UFE_CUDA(cudaFuncGetAttributes(&fa, k_ml_neumann));
    UFE_CUDA(cudaFuncGetAttributes(&fa, k_ml_final));
    UFE_CUDA(cudaFuncGetAttributes(&fa, k_ml_prolong));
  }
}

void ml_coarse_solve(const Bddc& B, const double* gC, double* uc, const PcgScalars* sc, cudaStream_t s) {
  const MultiLevel& L = B.ml;
  const MlMeta M = meta_of(L);
  const size_t s1 = (size_t)(pad4(L.max_n) + pad4(L.max_nI)) * 8;
  const size_t s2 = (size_t)2 * pad4(L.max_nG) * 8;
  const size_t s4 = (size_t)(pad4(L.max_nG) + 2 * pad4(L.max_nI)) * 8;
  k_ml_interior<<<L.n2, 256, s1, s>>>(M, B.cpos.p, B.coarse_nn.p, gC, sc);
  UFE_CHECK_LAUNCH();
  k_ml_neumann<<<L.n2, 256, s2, s>>>(M, sc);
  UFE_CHECK_LAUNCH();
  const size_t s34 = (size_t)(L.ld3 + pad4(L.max_nC) + pad4(L.max_nG)) * 8;
  if (L.n3 > 0 && s34 <= kFusedCoarse3Smem) {
    k_ml_coarse3<<<L.n2, 256, s34, s>>>(M, L.n3, L.ld3, L.A3inv.p, L.cpos3.p, L.nn3.p, sc);
    UFE_CHECK_LAUNCH();
  } else if (L.n3 > 0) {
    dense_coarse_gemv(L.n3, L.ld3, L.A3inv.p, L.cpos3.p, L.nn3.p, L.g3.p, L.u3.p, sc, s);
    k_ml_prolong<<<L.n2, 256, (size_t)(pad4(L.max_nC) + pad4(L.max_nG)) * 8, s>>>(M, sc);
    UFE_CHECK_LAUNCH();
  }
  k_ml_final<<<L.n2, 256, s4, s>>>(M, uc, sc);
  UFE_CHECK_LAUNCH();
}

}  // namespace ufe
