// Cut-cell integration and right-hand side (Sect. 2.2).
//
// Each cube is split into the 6 Kuhn tetrahedra v000 -> v000+e_a -> v000+e_a+e_b
// -> v111; the level set is linear on each tetrahedron and the part {phi < 0} is
// cut out with the edge crossing points.  1 or 3 inside vertices leave a tet or a
// prism, 2 leave a prism; prisms are split into 3 tets.  The boundary facet is a
// triangle or a planar quad (2 triangles) with normal grad(phi)/|grad(phi)|.
// Poisson: every volume integrand (grad N_a . grad N_b, degree <= 4, and f_h N_a,
// degree <= 6) is a combination of the 27 separable moments
// int q_i(x) q_j(y) q_k(z), q in {(1-t)^2, t(1-t), t^2}, accumulated with the degree-7
// Grundmann-Moeller tet rule (35 points); elasticity uses the degree-5 rule (15 points)
// for its degree-4 gradient products; facets use the degree-7 triangle rule.  Every
// integral is therefore exact up to rounding.  The rules are generated on the host from the published
// formula of Grundmann & Moeller (1978) and kept in constant memory.
//
// One warp per cut cell (see k_integrate_cut).
#include <cmath>
#include <functional>
#include <mutex>
#include <vector>

#include "q1.cuh"
#include "ufe_internal.cuh"

namespace ufe {

constexpr int kTetPts = 35, kTriPts = 20, kTet5Pts = 15;
__constant__ double c_tet_bary[kTetPts * 4];
__constant__ double c_tet_w[kTetPts];
__constant__ double c_tet5_bary[kTet5Pts * 4];
__constant__ double c_tet5_w[kTet5Pts];
__constant__ double c_tri_bary[kTriPts * 3];
__constant__ double c_tri_w[kTriPts];
// moments int q_i(x) q_j(y) q_k(z) over each whole Kuhn tet (unit-cube coordinates),
// q in {(1-t)^2, t(1-t), t^2}: added once for a Kuhn tet that lies inside the domain
__constant__ double c_kuhn_mom[6][27];

// Grundmann-Moeller rule of degree 2s+1 on the n-simplex; weights rescaled to sum to 1.
static void gm_rule(int n, int s, std::vector<double>& bary, std::vector<double>& w) {
  const int d = 2 * s + 1;
  auto fact = [](int k) {
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
  };
  bary.clear();
  w.clear();
  for (int i = 0; i <= s; ++i) {
    const int denom = d + n - 2 * i;
    const double wt = ((i % 2) ? -1.0 : 1.0) * std::ldexp(1.0, -2 * s) * std::pow((double)denom, d) /
                      (fact(i) * fact(d + n - i)) * fact(n);
    // all (n+1)-tuples beta >= 0 with |beta| = s - i
    std::vector<int> beta(n + 1, 0);
    std::function<void(int, int)> rec = [&](int pos, int remaining) {
      if (pos == n) {
        beta[n] = remaining;
        for (int j = 0; j <= n; ++j) bary.push_back((2.0 * beta[j] + 1.0) / denom);
        w.push_back(wt);
        return;
      }
      for (int v = 0; v <= remaining; ++v) {
        beta[pos] = v;
        rec(pos + 1, remaining - v);
      }
    };
    rec(0, s - i);
  }
}

void ensure_constants() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  for (int d : done)
    if (d == dev) return;
  std::vector<double> b, w;
  gm_rule(3, 3, b, w);
  UFE_REQUIRE((int)w.size() == kTetPts, UFE_ERR_CUDA, "tet rule size");
  UFE_CUDA(cudaMemcpyToSymbol(c_tet_bary, b.data(), b.size() * sizeof(double)));
  UFE_CUDA(cudaMemcpyToSymbol(c_tet_w, w.data(), w.size() * sizeof(double)));
  gm_rule(3, 2, b, w);
  UFE_REQUIRE((int)w.size() == kTet5Pts, UFE_ERR_CUDA, "tet degree-5 rule size");
  UFE_CUDA(cudaMemcpyToSymbol(c_tet5_bary, b.data(), b.size() * sizeof(double)));
  UFE_CUDA(cudaMemcpyToSymbol(c_tet5_w, w.data(), w.size() * sizeof(double)));
  {
    // Kuhn tet t: v000 -> v000 + e_a -> v000 + e_a + e_b -> v111 (the kernel's order),
    // integrated with the same 35-point rule (degree 7: exact for these degree-6 moments)
    std::vector<double> bt, wt;
    gm_rule(3, 3, bt, wt);
    const int ax0[6] = {0, 0, 1, 1, 2, 2}, ax1[6] = {1, 2, 0, 2, 0, 1};
    double mom[6][27];
    for (int t = 0; t < 6; ++t) {
      const int vid[4] = {0, 1 << ax0[t], (1 << ax0[t]) | (1 << ax1[t]), 7};
      for (int e = 0; e < 27; ++e) mom[t][e] = 0.0;
      for (size_t qp = 0; qp < wt.size(); ++qp) {
        double x[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < 4; ++m)
          for (int d = 0; d < 3; ++d) x[d] += bt[qp * 4 + m] * (double)((vid[m] >> d) & 1);
        double qv[3][3];
        for (int d = 0; d < 3; ++d) {
          const double u = 1.0 - x[d];
          qv[d][0] = u * u;
          qv[d][1] = x[d] * u;
          qv[d][2] = x[d] * x[d];
        }
        const double wq = wt[qp] / 6.0;   // every Kuhn tet has volume 1/6
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) mom[t][9 * i + 3 * j + k] += wq * qv[0][i] * qv[1][j] * qv[2][k];
      }
    }
    UFE_CUDA(cudaMemcpyToSymbol(c_kuhn_mom, mom, sizeof(mom)));
  }
  gm_rule(2, 3, b, w);
  UFE_REQUIRE((int)w.size() == kTriPts, UFE_ERR_CUDA, "triangle rule size");
  UFE_CUDA(cudaMemcpyToSymbol(c_tri_bary, b.data(), b.size() * sizeof(double)));
  UFE_CUDA(cudaMemcpyToSymbol(c_tri_w, w.data(), w.size() * sizeof(double)));
  done.push_back(dev);
}


struct Vec3 {
  double x, y, z;
};
__device__ __forceinline__ Vec3 lerp_cross(const Vec3& pu, const Vec3& pv, double fu, double fv) {
  const double t = fu / (fu - fv);
  return {pu.x + t * (pv.x - pu.x), pu.y + t * (pv.y - pu.y), pu.z + t * (pv.z - pu.z)};
}

// Per cut cell, six lanes clip the six Kuhn tets and write the sub-tets and
// boundary triangles into shared memory; then all 32 lanes of the warp share the
// (sub-tet, point) and (triangle, point) work items and the 45 partial sums are
// reduced with warp shuffles.
constexpr int kWarpsPerBlock = 8;
constexpr int kMaxSubTets = 18, kMaxTris = 12;

struct CellGeom {
  double tet[kMaxSubTets][12];   // 4 vertices x (x, y, z), unit-cube coordinates
  double tri[kMaxTris][12];      // 3 vertices x (x, y, z) + unit normal
  int n_tet, n_tri;
};

__device__ __forceinline__ void put3(double* d, const Vec3& v) {
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
}

// clip one Kuhn tet: writes its sub-tets / triangles into local arrays; returns counts
__device__ void clip_tet(const Vec3 P[4], const double F[4], double st[3][12], int& nst, double tr[2][12], int& ntr) {
  nst = 0;
  ntr = 0;
  int neg[4], pos[4], nn = 0, np = 0;
  for (int m = 0; m < 4; ++m) {
    if (F[m] < 0.0)
      neg[nn++] = m;
    else
      pos[np++] = m;
  }
  if (nn == 0) return;
  auto tet = [&](const Vec3& A, const Vec3& B, const Vec3& C, const Vec3& D) {
    put3(st[nst] + 0, A);
    put3(st[nst] + 3, B);
    put3(st[nst] + 6, C);
    put3(st[nst] + 9, D);
    ++nst;
  };
  if (nn == 4) {
    tet(P[0], P[1], P[2], P[3]);
    return;
  }
  // gradient of the linear level set on the tet (Cramer's rule); unit normal
  const double d1x = P[1].x - P[0].x, d1y = P[1].y - P[0].y, d1z = P[1].z - P[0].z;
  const double d2x = P[2].x - P[0].x, d2y = P[2].y - P[0].y, d2z = P[2].z - P[0].z;
  const double d3x = P[3].x - P[0].x, d3y = P[3].y - P[0].y, d3z = P[3].z - P[0].z;
  const double r1 = F[1] - F[0], r2 = F[2] - F[0], r3 = F[3] - F[0];
  const double det = d1x * (d2y * d3z - d2z * d3y) - d1y * (d2x * d3z - d2z * d3x) + d1z * (d2x * d3y - d2y * d3x);
  const double gx = (r1 * (d2y * d3z - d2z * d3y) - d1y * (r2 * d3z - d2z * r3) + d1z * (r2 * d3y - d2y * r3)) / det;
  const double gy = (d1x * (r2 * d3z - d2z * r3) - r1 * (d2x * d3z - d2z * d3x) + d1z * (d2x * r3 - r2 * d3x)) / det;
  const double gz = (d1x * (d2y * r3 - r2 * d3y) - d1y * (d2x * r3 - r2 * d3x) + r1 * (d2x * d3y - d2y * d3x)) / det;
  const double gn = sqrt(gx * gx + gy * gy + gz * gz);
  const Vec3 nrm = {gx / gn, gy / gn, gz / gn};
  auto tri = [&](const Vec3& A, const Vec3& B, const Vec3& C) {
    put3(tr[ntr] + 0, A);
    put3(tr[ntr] + 3, B);
    put3(tr[ntr] + 6, C);
    put3(tr[ntr] + 9, nrm);
    ++ntr;
  };
  if (nn == 1) {
    const int a = neg[0], b = pos[0], c = pos[1], d = pos[2];
    const Vec3 pab = lerp_cross(P[a], P[b], F[a], F[b]);
    const Vec3 pac = lerp_cross(P[a], P[c], F[a], F[c]);
    const Vec3 pad = lerp_cross(P[a], P[d], F[a], F[d]);
    tet(P[a], pab, pac, pad);
    tri(pab, pac, pad);
  } else if (nn == 3) {
    const int a = neg[0], b = neg[1], c = neg[2], d = pos[0];
    const Vec3 pad = lerp_cross(P[a], P[d], F[a], F[d]);
    const Vec3 pbd = lerp_cross(P[b], P[d], F[b], F[d]);
    const Vec3 pcd = lerp_cross(P[c], P[d], F[c], F[d]);
    tet(P[a], P[b], P[c], pad);
    tet(P[b], P[c], pad, pbd);
    tet(P[c], pad, pbd, pcd);
    tri(pad, pbd, pcd);
  } else {
    const int a = neg[0], b = neg[1], c = pos[0], d = pos[1];
    const Vec3 pac = lerp_cross(P[a], P[c], F[a], F[c]);
    const Vec3 pad = lerp_cross(P[a], P[d], F[a], F[d]);
    const Vec3 pbc = lerp_cross(P[b], P[c], F[b], F[c]);
    const Vec3 pbd = lerp_cross(P[b], P[d], F[b], F[d]);
    tet(P[a], pac, pad, P[b]);
    tet(pac, pad, P[b], pbc);
    tet(pad, P[b], pbc, pbd);
    tri(pac, pad, pbd);
    tri(pac, pbd, pbc);
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2)
k_integrate_cut(GridGeom g, int64_t n_cut, const int32_t* __restrict__ cut_cells, const double* __restrict__ phi,
                const double* __restrict__ f, const double* __restrict__ q, double* __restrict__ K_cut,
                double* __restrict__ load_cut, double* __restrict__ eta) {
  __shared__ double s_tet[kTetPts * 5];   // 4 barycentric + weight
  __shared__ double s_tri[kTriPts * 4];
  __shared__ CellGeom geo[kWarpsPerBlock];
  __shared__ double s_f[kWarpsPerBlock][8];
  __shared__ double s_q[kWarpsPerBlock][8][3];
  for (int e = threadIdx.x; e < kTetPts; e += blockDim.x) {
    for (int c = 0; c < 4; ++c) s_tet[e * 5 + c] = c_tet_bary[e * 4 + c];
    s_tet[e * 5 + 4] = c_tet_w[e];
  }
  for (int e = threadIdx.x; e < kTriPts; e += blockDim.x) {
    for (int c = 0; c < 3; ++c) s_tri[e * 4 + c] = c_tri_bary[e * 3 + c];
    s_tri[e * 4 + 3] = c_tri_w[e];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t kc = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  const bool valid = kc < n_cut;
  CellGeom& G = geo[warp];
  int ntet_l = 0, ntri_l = 0;
  bool full = false;   // this lane's Kuhn tet lies inside: its moments come from the table
  double st[3][12], tr[2][12];
  if (valid) {
    const int64_t c = cut_cells[kc];
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((int64_t)g.nx * g.ny));
    if (lane < 8) {
      const int64_t v = g.node(i + (lane & 1), j + ((lane >> 1) & 1), k + (lane >> 2));
      s_f[warp][lane] = f ? f[v] : 0.0;
      for (int d = 0; d < 3; ++d) s_q[warp][lane][d] = q ? q[3 * v + d] : 0.0;
    }
    if (lane < 6) {
      const int ax0[6] = {0, 0, 1, 1, 2, 2};
      const int ax1[6] = {1, 2, 0, 2, 0, 1};
      const int vid[4] = {0, 1 << ax0[lane], (1 << ax0[lane]) | (1 << ax1[lane]), 7};
      Vec3 P[4];
      double F[4];
      for (int m = 0; m < 4; ++m) {
        P[m] = {(double)(vid[m] & 1), (double)((vid[m] >> 1) & 1), (double)(vid[m] >> 2)};
        F[m] = phi[g.node(i + (vid[m] & 1), j + ((vid[m] >> 1) & 1), k + (vid[m] >> 2))];
      }
      full = F[0] < 0.0 && F[1] < 0.0 && F[2] < 0.0 && F[3] < 0.0;
      if (!full) clip_tet(P, F, st, ntet_l, tr, ntri_l);
    }
  }
  const unsigned full_mask = __ballot_sync(0xffffffffu, full);
  // compact the per-tet pieces of lanes 0..5 into the warp's shared geometry
  int off_t = ntet_l, off_r = ntri_l;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int a = __shfl_up_sync(0xffffffffu, off_t, o), b = __shfl_up_sync(0xffffffffu, off_r, o);
    if (lane >= o) {
      off_t += a;
      off_r += b;
    }
  }
  const int tot_t = __shfl_sync(0xffffffffu, off_t, 7), tot_r = __shfl_sync(0xffffffffu, off_r, 7);
  off_t -= ntet_l;
  off_r -= ntri_l;
  for (int a = 0; a < ntet_l; ++a)
    for (int e = 0; e < 12; ++e) G.tet[off_t + a][e] = st[a][e];
  for (int a = 0; a < ntri_l; ++a)
    for (int e = 0; e < 12; ++e) G.tri[off_r + a][e] = tr[a][e];
  if (lane == 0) {
    G.n_tet = tot_t;
    G.n_tri = (q != nullptr) ? tot_r : 0;
  }
  __syncthreads();
  // Every integrand is a polynomial in the separable basis q_i(x) q_j(y) q_k(z),
  // q_0 = (1-t)^2, q_1 = t (1-t), q_2 = t^2 (unit-cube coordinates), so the lanes
  // accumulate the 27 moments M_ijk = int q_i(x) q_j(y) q_k(z) over the sub-tets
  // (degree 6: the 35-point rule is exact) and, with a flux, the 8 facet loads;
  // K, the source load and the volume fraction follow from the moments at the end.
  constexpr int kMom = 27, kVals = kMom + 8;
  double acc[kVals];
#pragma unroll
  for (int e = 0; e < kVals; ++e) acc[e] = 0.0;
  const double h = g.h, h3 = h * h * h, h2 = h * h;
  if (valid) {
    const int n_v = G.n_tet * kTetPts;
    const int n_all = n_v + G.n_tri * kTriPts;
    for (int it = lane; it < n_all; it += 32) {
      if (it < n_v) {
        const double* T = G.tet[it / kTetPts];
        const double* R = s_tet + (it % kTetPts) * 5;
        const double ux = T[3] - T[0], uy = T[4] - T[1], uz = T[5] - T[2];
        const double vx = T[6] - T[0], vy = T[7] - T[1], vz = T[8] - T[2];
        const double wx = T[9] - T[0], wy = T[10] - T[1], wz = T[11] - T[2];
        const double vol =
            fabs(ux * (vy * wz - vz * wy) - uy * (vx * wz - vz * wx) + uz * (vx * wy - vy * wx)) / 6.0;
        const double px = R[0] * T[0] + R[1] * T[3] + R[2] * T[6] + R[3] * T[9];
        const double py = R[0] * T[1] + R[1] * T[4] + R[2] * T[7] + R[3] * T[10];
        const double pz = R[0] * T[2] + R[1] * T[5] + R[2] * T[8] + R[3] * T[11];
        const double wq = R[4] * vol;
        const double mx = 1.0 - px, my = 1.0 - py, mz = 1.0 - pz;
        const double qx[3] = {mx * mx, px * mx, px * px};
        const double qy[3] = {my * my, py * my, py * py};
        const double qz[3] = {wq * mz * mz, wq * pz * mz, wq * pz * pz};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const double xy = qx[i] * qy[j];
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[9 * i + 3 * j + k] = fma(xy, qz[k], acc[9 * i + 3 * j + k]);
          }
      } else {
        const int r = it - n_v;
        const double* T = G.tri[r / kTriPts];
        const double* R = s_tri + (r % kTriPts) * 4;
        const double ux = T[3] - T[0], uy = T[4] - T[1], uz = T[5] - T[2];
        const double vx = T[6] - T[0], vy = T[7] - T[1], vz = T[8] - T[2];
        const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
        const double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
        const double px = R[0] * T[0] + R[1] * T[3] + R[2] * T[6];
        const double py = R[0] * T[1] + R[1] * T[4] + R[2] * T[7];
        const double pz = R[0] * T[2] + R[1] * T[5] + R[2] * T[8];
        const double wq = R[3] * area;
        double N[8];
        q1_shape(px, py, pz, N);
        double qxv = 0, qyv = 0, qzv = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          qxv += N[a] * s_q[warp][a][0];
          qyv += N[a] * s_q[warp][a][1];
          qzv += N[a] * s_q[warp][a][2];
        }
        const double gnv = qxv * T[9] + qyv * T[10] + qzv * T[11];
#pragma unroll
        for (int a = 0; a < 8; ++a) acc[kMom + a] += wq * gnv * N[a] * h2;
      }
    }
  }
  // moments: reduce-scatter over the warp (fixed butterfly), after the five levels
  // lane l holds the warp total of moment l (27 .. 31 are zero padding)
  double v[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) v[e] = e < kMom ? acc[e] : 0.0;
#pragma unroll
  for (int o = 16, w = 16; o > 0; o >>= 1, w >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const double send = up ? v[i] : v[i + w];
      const double keep = up ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  // facet loads (with a flux only): plain butterfly sums, every lane gets all eight
  double fl = 0.0;
  if (q != nullptr) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      double t = acc[kMom + a];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == a) fl = t;
    }
  }
  if (lane < kMom)
    for (int t = 0; t < 6; ++t)
      if (full_mask & (1u << t)) v[0] += c_kuhn_mom[t][lane];
  __shared__ double s_val[kWarpsPerBlock][32];
  s_val[warp][lane] = v[0];
  __syncwarp();
  if (valid) {
    const double* M = s_val[warp];
    // K_ab = h sum_d s(a_d) s(b_d) int prod_{d' != d} l_a l_b, with l_a l_b = q_{a + b}
    // and int q_j(y) q_k(z) = sum_i c_i M_ijk, c = (1, 2, 1) (q_0 + 2 q_1 + q_2 = 1)
    for (int e = lane; e < 64; e += 32) {
      const int a = e >> 3, bb = e & 7;
      const int sx = (a & 1) + (bb & 1), sy = ((a >> 1) & 1) + ((bb >> 1) & 1), sz = (a >> 2) + (bb >> 2);
      const double fx = sx == 1 ? -1.0 : 1.0, fy = sy == 1 ? -1.0 : 1.0, fz = sz == 1 ? -1.0 : 1.0;
      const double Sx = M[0 + 3 * sy + sz] + 2.0 * M[9 + 3 * sy + sz] + M[18 + 3 * sy + sz];
      const double Sy = M[9 * sx + 0 + sz] + 2.0 * M[9 * sx + 3 + sz] + M[9 * sx + 6 + sz];
      const double Sz = M[9 * sx + 3 * sy + 0] + 2.0 * M[9 * sx + 3 * sy + 1] + M[9 * sx + 3 * sy + 2];
      K_cut[kc * 64 + e] = h * (fx * Sx + fy * Sy + fz * Sz);
    }
    if (lane < 8) {
      // source load: h^3 sum_b f_b int N_a N_b, N_a N_b = q_{a_x + b_x} q_{a_y + b_y} q_{a_z + b_z}
      const int a = lane;
      double l = 0.0;
      for (int bb = 0; bb < 8; ++bb) {
        const int i = (a & 1) + (bb & 1), j = ((a >> 1) & 1) + ((bb >> 1) & 1), k = (a >> 2) + (bb >> 2);
        l = fma(s_f[warp][bb], M[9 * i + 3 * j + k], l);
      }
      load_cut[kc * 8 + a] = h3 * l + fl;
    } else if (lane == 8) {
      const double c[3] = {1.0, 2.0, 1.0};
      double vol = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          for (int k = 0; k < 3; ++k) vol = fma(c[i] * c[j] * c[k], M[9 * i + 3 * j + k], vol);
      eta[kc] = vol;
    }
  }
}

// b = sum_e load_e - A_FC g_C  over the free DOFs (one thread per DOF, cells in a fixed order)
__global__ void k_rhs(GridGeom g, int64_t n_dof, const int32_t* __restrict__ node_of_dof,
                      const int32_t* __restrict__ dof_of_node, const uint8_t* __restrict__ cell_type,
                      const int32_t* __restrict__ cut_index, const double* __restrict__ K_cut,
                      const double* __restrict__ load_cut, const double* __restrict__ kappa,
                      const double* __restrict__ f, const double* __restrict__ gval,
                      const uint8_t* __restrict__ node_flags, double* __restrict__ b) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof) return;
  const int64_t v = node_of_dof[d];
  const int i = (int)(v % (g.nx + 1)), j = (int)((v / (g.nx + 1)) % (g.ny + 1));
  const int k = (int)(v / ((int64_t)(g.nx + 1) * (g.ny + 1)));
  const double h = g.h, h3 = h * h * h;
  double sum = 0.0;
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        const int ci = i + di, cj = j + dj, ck = k + dk;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx || cj >= g.ny || ck >= g.nz) continue;
        const int64_t c = g.cell(ci, cj, ck);
        const uint8_t t = cell_type[c];
        if (t == UFE_CELL_EXTERNAL) continue;
        const int a = (-di) + 2 * (-dj) + 4 * (-dk);
        const int32_t cx = t == UFE_CELL_CUT ? cut_index[c] : -1;
        if (t == UFE_CELL_INTERNAL) {
          if (f) {
            double s = 0.0;
            for (int bb = 0; bb < 8; ++bb)
              s += q1_mhat(a, bb) * f[g.node(ci + (bb & 1), cj + ((bb >> 1) & 1), ck + (bb >> 2))];
            sum += h3 * s;
          }
        } else {
          sum += load_cut[(int64_t)cx * 8 + a];
        }
        if (gval) {
          const double kap = kappa ? kappa[c] : 1.0;
          for (int bb = 0; bb < 8; ++bb) {
            const int64_t vb = g.node(ci + (bb & 1), cj + ((bb >> 1) & 1), ck + (bb >> 2));
            // constrained = active node that is not a free DOF
            if (dof_of_node[vb] >= 0 || !(node_flags[vb] & 1)) continue;
            const double kab = t == UFE_CELL_INTERNAL ? h * q1_khat(a, bb) : K_cut[(int64_t)cx * 64 + a * 8 + bb];
            sum -= kap * kab * gval[vb];
          }
        }
      }
  b[d] = sum;
}

__global__ void k_cut_list(int64_t n, const int32_t* __restrict__ cut_index, int32_t* __restrict__ cut_cells) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int32_t k = cut_index[c];
  if (k >= 0) cut_cells[k] = (int32_t)c;
}
void launch_cut_list(const Mesh& m, cudaStream_t s) {
  k_cut_list<<<grid_for(m.g.n_cells(), 256), 256, 0, s>>>(m.g.n_cells(), m.cut_index.p, m.cut_cells.p);
  UFE_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Weak Dirichlet data on the unfitted boundary (Nitsche, Sect. 2.2).  Every cut cell
// gains h (beta M - C - C^T) in its matrix and h (beta M g - C^T g) in its load, with
// the unit-cube facet forms
//   M_ab = int N_a N_b dS,  C_ab = int N_a (n . grad N_b) dS,  B_ab = int (n . grad N_a)(n . grad N_b) dS
// over the cell's boundary triangles (the same marching-tetrahedra surface as the
// Neumann data), g the Q1 interpolant of the nodal Dirichlet values, and beta = 2 C_e
// (unit-cube; C_e the largest eigenvalue of B x = lambda D x on the complement of the
// constants, D the cut-cell stiffness, Eq. local-eigenvals).  C_e is computed after a
// symmetric Jacobi scaling by diag(D)^-1/2, in an orthonormal (Householder) basis of the
// complement of the scaled kernel vector, by a Cholesky reduction to a 7 x 7 symmetric
// matrix and cyclic Jacobi rotations.
//
// One warp per cut cell.  Six lanes clip the Kuhn tets (the triangles are kept); the
// facet points are taken 32 at a time: each lane evaluates N and n . grad N of one
// point into shared memory, then each lane accumulates its entries of M, B (36 unique
// each) and C (64) over the 32 points in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kNiWarps = 4;
constexpr int kNiEntries = 36 + 36 + 64;
constexpr int kNiPerLane = (kNiEntries + 31) / 32;

// largest eigenvalue of B x = lambda D x on the complement of the constants (8 x 8,
// row-major, both symmetric with the constants in their kernel); w: kNiScratch doubles
constexpr int kNiScratch = 56 + 4 * 49 + 8;
__device__ double nitsche_constant(const double* __restrict__ D, const double* __restrict__ B, double* w) {
  double* V = w;            // 8 x 7 orthonormal basis of the complement of the scaled kernel vector
  double* L = w + 56;       // 7 x 7: S D S in the basis, then its Cholesky factor (lower)
  double* B7 = w + 105;     // 7 x 7: S B S in the basis
  double* Y = w + 154;      // 7 x 7: L^-1 B7
  double* G = w + 203;      // 7 x 7: L^-1 B7 L^-T
  double* T = w + 252;      // 8
  double s[8], v[8];
  double kn = 0.0;
  for (int a = 0; a < 8; ++a) {
    s[a] = 1.0 / sqrt(D[a * 8 + a]);
    v[a] = sqrt(D[a * 8 + a]);   // kernel of S D S: S^-1 (1, ..., 1)
    kn += D[a * 8 + a];
  }
  kn = sqrt(kn);
  for (int a = 0; a < 8; ++a) v[a] /= kn;
  v[0] += v[0] >= 0.0 ? 1.0 : -1.0;   // Householder vector: H maps the kernel vector to -+e_0
  double vv = 0.0;
  for (int a = 0; a < 8; ++a) vv += v[a] * v[a];
  for (int a = 0; a < 8; ++a)
    for (int c = 1; c < 8; ++c) V[a * 7 + (c - 1)] = (a == c ? 1.0 : 0.0) - 2.0 * v[a] * v[c] / vv;
  // L = V^T S D S V, B7 = V^T S B S V (each entry once, mirrored)
  for (int pass = 0; pass < 2; ++pass) {
    const double* X = pass == 0 ? D : B;
    double* Z = pass == 0 ? L : B7;
    for (int j = 0; j < 7; ++j) {
      for (int a = 0; a < 8; ++a) {
        double t = 0.0;
        for (int b = 0; b < 8; ++b) t += X[a * 8 + b] * (s[b] * V[b * 7 + j]);
        T[a] = s[a] * t;
      }
      for (int i = j; i < 7; ++i) {
        double t = 0.0;
        for (int a = 0; a < 8; ++a) t += V[a * 7 + i] * T[a];
        Z[i * 7 + j] = t;
        Z[j * 7 + i] = t;
      }
    }
  }
  // Cholesky: L (lower triangle) with L L^T = the scaled D in the basis
  for (int j = 0; j < 7; ++j) {
    double d = L[j * 7 + j];
    for (int m = 0; m < j; ++m) d -= L[j * 7 + m] * L[j * 7 + m];
    if (!(d > 0.0)) return nan("");
    d = sqrt(d);
    L[j * 7 + j] = d;
    for (int i = j + 1; i < 7; ++i) {
      double t = L[i * 7 + j];
      for (int m = 0; m < j; ++m) t -= L[i * 7 + m] * L[j * 7 + m];
      L[i * 7 + j] = t / d;
    }
  }
  // Y = L^-1 B7, G = L^-1 Y^T (= L^-1 B7 L^-T, B7 symmetric), column by column
  for (int c = 0; c < 7; ++c)
    for (int i = 0; i < 7; ++i) {
      double t = B7[i * 7 + c];
      for (int m = 0; m < i; ++m) t -= L[i * 7 + m] * Y[m * 7 + c];
      Y[i * 7 + c] = t / L[i * 7 + i];
    }
  for (int c = 0; c < 7; ++c)
    for (int i = 0; i < 7; ++i) {
      double t = Y[c * 7 + i];
      for (int m = 0; m < i; ++m) t -= L[i * 7 + m] * G[m * 7 + c];
      G[i * 7 + c] = t / L[i * 7 + i];
    }
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < i; ++j) {
      const double t = 0.5 * (G[i * 7 + j] + G[j * 7 + i]);
      G[i * 7 + j] = t;
      G[j * 7 + i] = t;
    }
  // cyclic Jacobi rotations (bounded number of sweeps)
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < 7; ++i)
      for (int j = 0; j < 7; ++j) {
        tot += G[i * 7 + j] * G[i * 7 + j];
        if (i != j) off += G[i * 7 + j] * G[i * 7 + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < 6; ++p)
      for (int q = p + 1; q < 7; ++q) {
        const double apq = G[p * 7 + q];
        if (apq == 0.0) continue;
        const double theta = (G[q * 7 + q] - G[p * 7 + p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int r = 0; r < 7; ++r) {   // G <- G J (columns p, q)
          const double gp = G[r * 7 + p], gq = G[r * 7 + q];
          G[r * 7 + p] = c * gp - sn * gq;
          G[r * 7 + q] = sn * gp + c * gq;
        }
        for (int r = 0; r < 7; ++r) {   // G <- J^T G (rows p, q)
          const double gp = G[p * 7 + r], gq = G[q * 7 + r];
          G[p * 7 + r] = c * gp - sn * gq;
          G[q * 7 + r] = sn * gp + c * gq;
        }
      }
  }
  double lmax = G[0];
  for (int i = 1; i < 7; ++i) lmax = fmax(lmax, G[i * 7 + i]);
  return lmax;
}

__global__ void __launch_bounds__(kNiWarps * 32)
k_nitsche_cut(GridGeom g, int64_t n_cut, const int32_t* __restrict__ cut_cells, const double* __restrict__ phi,
              const double* __restrict__ gD, double* __restrict__ K_cut, double* __restrict__ load_cut,
              double* __restrict__ beta_out, int* __restrict__ status) {
  __shared__ double s_tri[kTriPts * 4];
  __shared__ double tris[kNiWarps][kMaxTris][12];
  __shared__ double s_pt[kNiWarps][32][17];
  __shared__ double s_mat[kNiWarps][kNiEntries];
  __shared__ double s_work[kNiWarps][64 + kNiScratch];
  __shared__ double s_beta[kNiWarps];
  for (int e = threadIdx.x; e < kTriPts; e += blockDim.x) {
    for (int c = 0; c < 3; ++c) s_tri[e * 4 + c] = c_tri_bary[e * 3 + c];
    s_tri[e * 4 + 3] = c_tri_w[e];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t kc = (int64_t)blockIdx.x * kNiWarps + warp;
  const bool valid = kc < n_cut;
  int ntri_l = 0;
  double st[3][12], tr[2][12];
  int cell_i = 0, cell_j = 0, cell_k = 0;
  if (valid) {
    const int64_t c = cut_cells[kc];
    cell_i = (int)(c % g.nx);
    cell_j = (int)((c / g.nx) % g.ny);
    cell_k = (int)(c / ((int64_t)g.nx * g.ny));
    if (lane < 6) {
      const int ax0[6] = {0, 0, 1, 1, 2, 2};
      const int ax1[6] = {1, 2, 0, 2, 0, 1};
      const int vid[4] = {0, 1 << ax0[lane], (1 << ax0[lane]) | (1 << ax1[lane]), 7};
      Vec3 P[4];
      double F[4];
      for (int m = 0; m < 4; ++m) {
        P[m] = {(double)(vid[m] & 1), (double)((vid[m] >> 1) & 1), (double)(vid[m] >> 2)};
        F[m] = phi[g.node(cell_i + (vid[m] & 1), cell_j + ((vid[m] >> 1) & 1), cell_k + (vid[m] >> 2))];
      }
      int nst = 0;
      const bool full = F[0] < 0.0 && F[1] < 0.0 && F[2] < 0.0 && F[3] < 0.0;
      if (!full) clip_tet(P, F, st, nst, tr, ntri_l);
    }
  }
  int off = ntri_l;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int a = __shfl_up_sync(0xffffffffu, off, o);
    if (lane >= o) off += a;
  }
  const int ntri = __shfl_sync(0xffffffffu, off, 7);
  off -= ntri_l;
  for (int a = 0; a < ntri_l; ++a)
    for (int e = 0; e < 12; ++e) tris[warp][off + a][e] = tr[a][e];
  __syncthreads();
  // entry e of this lane: M (0..35), B (36..71) as packed upper triangles, C (72..135) row-major
  int ea[kNiPerLane], eb[kNiPerLane], ek[kNiPerLane];
  double acc[kNiPerLane];
#pragma unroll
  for (int t = 0; t < kNiPerLane; ++t) {
    const int e = lane + 32 * t;
    acc[t] = 0.0;
    ek[t] = e < 36 ? 0 : (e < 72 ? 1 : (e < kNiEntries ? 2 : 3));
    int r = e < 36 ? e : (e < 72 ? e - 36 : e - 72);
    if (ek[t] <= 1) {
      int a = 0;
      while (r >= 8 - a) {
        r -= 8 - a;
        ++a;
      }
      ea[t] = a;
      eb[t] = a + r;
    } else {
      ea[t] = (r / 8) & 7;
      eb[t] = r % 8;
    }
  }
  const int npts = valid ? ntri * kTriPts : 0;
  for (int base = 0; base < npts; base += 32) {
    const int it = base + lane;
    double* P = s_pt[warp][lane];
    if (it < npts) {
      const double* T = tris[warp][it / kTriPts];
      const double* R = s_tri + (it % kTriPts) * 4;
      const double ux = T[3] - T[0], uy = T[4] - T[1], uz = T[5] - T[2];
      const double vx = T[6] - T[0], vy = T[7] - T[1], vz = T[8] - T[2];
      const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
      const double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
      const double px = R[0] * T[0] + R[1] * T[3] + R[2] * T[6];
      const double py = R[0] * T[1] + R[1] * T[4] + R[2] * T[7];
      const double pz = R[0] * T[2] + R[1] * T[5] + R[2] * T[8];
      double N[8], G[8][3];
      q1_shape_grad(px, py, pz, N, G);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        P[a] = N[a];
        P[8 + a] = G[a][0] * T[9] + G[a][1] * T[10] + G[a][2] * T[11];
      }
      P[16] = R[3] * area;
    } else {
      P[16] = 0.0;
    }
    __syncwarp();
    const int cnt = min(32, npts - base);
    for (int q = 0; q < cnt; ++q) {
      const double* Q = s_pt[warp][q];
      const double wq = Q[16];
#pragma unroll
      for (int t = 0; t < kNiPerLane; ++t) {
        const double x = ek[t] == 1 ? Q[8 + ea[t]] : Q[ea[t]];
        const double y = ek[t] == 0 ? Q[eb[t]] : Q[8 + eb[t]];
        if (ek[t] < 3) acc[t] = fma(wq * x, y, acc[t]);
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int t = 0; t < kNiPerLane; ++t)
    if (ek[t] < 3) s_mat[warp][lane + 32 * t] = acc[t];
  __syncwarp();
  const double h = g.h;
  if (valid && lane == 0) {
    double beta = 0.0;
    if (ntri > 0) {
      double* D = s_work[warp];
      double Bf[64];
      const double* M = s_mat[warp];
      for (int a = 0; a < 8; ++a)
        for (int b = a; b < 8; ++b) {
          const int pk = a * 8 - (a * (a - 1)) / 2 + (b - a);
          Bf[a * 8 + b] = Bf[b * 8 + a] = M[36 + pk];
        }
      bool any = false;
      for (int e = 0; e < 64; ++e) any = any || Bf[e] != 0.0;
      if (any) {
        for (int e = 0; e < 64; ++e) D[e] = K_cut[kc * 64 + e] / h;
        const double lam = nitsche_constant(D, Bf, s_work[warp] + 64);
        if (!(lam >= 0.0) || !isfinite(lam)) atomicOr(status, DEV_SINGULAR);
        beta = 2.0 * lam;
      }
    }
    s_beta[warp] = beta;
  }
  __syncwarp();
  if (!valid) return;
  const double beta = s_beta[warp];
  const double* M = s_mat[warp];
  const double* C = s_mat[warp] + 72;
  auto msym = [&](int a, int b) {
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    return M[a * 8 - (a * (a - 1)) / 2 + (b - a)];
  };
  for (int e = lane; e < 64; e += 32) {
    const int a = e >> 3, b = e & 7;
    K_cut[kc * 64 + e] += h * (beta * msym(a, b) - C[a * 8 + b] - C[b * 8 + a]);
  }
  if (lane < 8) {
    const int a = lane;
    double mg = 0.0, cg = 0.0;
    for (int b = 0; b < 8; ++b) {
      const double gb = gD[g.node(cell_i + (b & 1), cell_j + ((b >> 1) & 1), cell_k + (b >> 2))];
      mg += msym(a, b) * gb;
      cg += C[b * 8 + a] * gb;
    }
    load_cut[kc * 8 + a] += h * (beta * mg - cg);
  }
  if (lane == 0) beta_out[kc] = beta / h;
}

void system_build(System& sys, const double* kappa, const double* f, const double* q, const double* gval,
                  bool weak_dirichlet) {
  ensure_constants();
  Mesh& m = *sys.mesh;
  cudaStream_t s = sys.stream;
  const int64_t n_cut = m.n_cut;
  m.cut_cells.alloc(n_cut > 0 ? n_cut : 1, s);
  launch_cut_list(m, s);
  sys.K_cut.alloc((n_cut > 0 ? n_cut : 1) * 64, s);
  sys.load_cut.alloc((n_cut > 0 ? n_cut : 1) * 8, s);
  sys.eta.alloc(n_cut > 0 ? n_cut : 1, s);
  if (n_cut > 0) {
    TimedLaunch tl;
    tl.begin("integrate_cut", s);
    k_integrate_cut<<<grid_for(n_cut, kWarpsPerBlock), kWarpsPerBlock * 32, 0, s>>>(
        m.g, n_cut, m.cut_cells.p, m.phi.p, f, q, sys.K_cut.p, sys.load_cut.p, sys.eta.p);
    UFE_CHECK_LAUNCH();
    tl.end(s);
  }
  sys.nitsche = weak_dirichlet;
  if (weak_dirichlet) {
    UFE_REQUIRE(gval != nullptr && q == nullptr, UFE_ERR_INVALID_ARG,
                "weak Dirichlet data need nodal values and no Neumann flux");
    sys.beta.alloc(n_cut > 0 ? n_cut : 1, s);
    sys.beta.zero();
    if (n_cut > 0) {
      DBuf<int> st;
      st.alloc(1, s);
      st.zero();
      k_nitsche_cut<<<grid_for(n_cut, kNiWarps), kNiWarps * 32, 0, s>>>(m.g, n_cut, m.cut_cells.p, m.phi.p, gval,
                                                                        sys.K_cut.p, sys.load_cut.p, sys.beta.p,
                                                                        st.p);
      UFE_CHECK_LAUNCH();
      UFE_REQUIRE(scalar_to_host(st.p, s) == 0, UFE_ERR_SINGULAR_LOCAL,
                  "a cut cell's Nitsche eigenproblem has no positive largest eigenvalue");
    }
  }
  sys.gnode.alloc(m.g.n_nodes(), s);
  if (gval)
    UFE_CUDA(cudaMemcpyAsync(sys.gnode.p, gval, m.g.n_nodes() * 8, cudaMemcpyDeviceToDevice, s));
  else
    sys.gnode.zero();
  sys.fnode.alloc(m.g.n_nodes(), s);
  if (f)
    UFE_CUDA(cudaMemcpyAsync(sys.fnode.p, f, m.g.n_nodes() * 8, cudaMemcpyDeviceToDevice, s));
  else
    sys.fnode.zero();
  sys.b.alloc(m.n_dof, s);
  k_rhs<<<grid_for(m.n_dof, 128), 128, 0, s>>>(m.g, m.n_dof, m.node_of_dof.p, m.dof_of_node.p, m.cell_type.p,
                                               m.cut_index.p, sys.K_cut.p, sys.load_cut.p, kappa, f, gval,
                                               m.node_flags.p, sys.b.p);
  UFE_CHECK_LAUNCH();
}

void system_rebuild_rhs(System& sys) {
  Mesh& m = *sys.mesh;
  k_rhs<<<grid_for(m.n_dof, 128), 128, 0, sys.stream>>>(m.g, m.n_dof, m.node_of_dof.p, m.dof_of_node.p,
                                                        m.cell_type.p, m.cut_index.p, sys.K_cut.p, sys.load_cut.p,
                                                        sys.has_kappa ? sys.kappa.p : nullptr, sys.fnode.p,
                                                        sys.gnode.p, m.node_flags.p, sys.b.p);
  UFE_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// linear elasticity (vector Q1, 3 DOFs per node): 24 x 24 cut-cell matrices
// ---------------------------------------------------------------------------
// The element matrix is assembled from the gradient Gram matrix of the cut part
//   Gm[p][q] = int d_i N_a d_j N_b    (p = 3a + i, q = 3b + j; symmetric, 300 entries)
// as K[3a+i][3b+j] = lam Gm[3a+i][3b+j] + mu Gm[3a+j][3b+i] + delta_ij mu sum_d Gm[3a+d][3b+d].
// One warp per cut cell.  Each lane owns about ten entries of Gm and walks the
// quadrature points 32 at a time: first every lane evaluates the 24 gradients of
// one point into shared memory, then every lane accumulates its entries over the
// 32 points (fixed order, no cross-lane reduction of Gm).  Loads (body force with
// the 35-point rule, boundary traction sigma_h n with the facet rule) use per-lane
// partial sums reduced with shuffles, as in the Poisson kernel.
constexpr int kElWarps = 4;
constexpr int kGram = 300;
constexpr int kGramPerLane = (kGram + 31) / 32;

__device__ __forceinline__ int gram_index(int p, int q) {
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
  return p * 24 - (p * (p - 1)) / 2 + (q - p);
}

__global__ void __launch_bounds__(kElWarps * 32)
k_integrate_cut_el(GridGeom g, int64_t n_cut, const int32_t* __restrict__ cut_cells, const double* __restrict__ phi,
                   const double* __restrict__ f, const double* __restrict__ sig, double lam, double mu,
                   double* __restrict__ K_cut, double* __restrict__ load_cut, double* __restrict__ eta) {
  __shared__ double s_tet[kTetPts * 5];
  __shared__ double s_tet5[kTet5Pts * 5];
  __shared__ double s_tri[kTriPts * 4];
  __shared__ uint8_t s_gp[kGram], s_gq[kGram];
  __shared__ CellGeom geo[kElWarps];
  __shared__ double s_f[kElWarps][8][3];
  __shared__ double s_s[kElWarps][8][9];
  __shared__ double s_pt[kElWarps][32 * 25];   // a chunk of points: 24 gradients + weight; later Gm
  for (int e = threadIdx.x; e < kTetPts; e += blockDim.x) {
    for (int c = 0; c < 4; ++c) s_tet[e * 5 + c] = c_tet_bary[e * 4 + c];
    s_tet[e * 5 + 4] = c_tet_w[e];
  }
  for (int e = threadIdx.x; e < kTet5Pts; e += blockDim.x) {
    for (int c = 0; c < 4; ++c) s_tet5[e * 5 + c] = c_tet5_bary[e * 4 + c];
    s_tet5[e * 5 + 4] = c_tet5_w[e];
  }
  for (int e = threadIdx.x; e < kTriPts; e += blockDim.x) {
    for (int c = 0; c < 3; ++c) s_tri[e * 4 + c] = c_tri_bary[e * 3 + c];
    s_tri[e * 4 + 3] = c_tri_w[e];
  }
  if (threadIdx.x < 24) {
    const int p = threadIdx.x;
    for (int q = p; q < 24; ++q) {
      const int e = gram_index(p, q);
      s_gp[e] = (uint8_t)p;
      s_gq[e] = (uint8_t)q;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t kc = (int64_t)blockIdx.x * kElWarps + warp;
  const bool valid = kc < n_cut;
  CellGeom& G = geo[warp];
  int ntet_l = 0, ntri_l = 0;
  double st[3][12], tr[2][12];
  if (valid) {
    const int64_t c = cut_cells[kc];
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((int64_t)g.nx * g.ny));
    if (lane < 8) {
      const int64_t v = g.node(i + (lane & 1), j + ((lane >> 1) & 1), k + (lane >> 2));
      for (int d = 0; d < 3; ++d) s_f[warp][lane][d] = f ? f[3 * v + d] : 0.0;
      for (int d = 0; d < 9; ++d) s_s[warp][lane][d] = sig ? sig[9 * v + d] : 0.0;
    }
    if (lane < 6) {
      const int ax0[6] = {0, 0, 1, 1, 2, 2};
      const int ax1[6] = {1, 2, 0, 2, 0, 1};
      const int vid[4] = {0, 1 << ax0[lane], (1 << ax0[lane]) | (1 << ax1[lane]), 7};
      Vec3 P[4];
      double F[4];
      for (int m = 0; m < 4; ++m) {
        P[m] = {(double)(vid[m] & 1), (double)((vid[m] >> 1) & 1), (double)(vid[m] >> 2)};
        F[m] = phi[g.node(i + (vid[m] & 1), j + ((vid[m] >> 1) & 1), k + (vid[m] >> 2))];
      }
      clip_tet(P, F, st, ntet_l, tr, ntri_l);
    }
  }
  int off_t = ntet_l, off_r = ntri_l;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int a = __shfl_up_sync(0xffffffffu, off_t, o), b = __shfl_up_sync(0xffffffffu, off_r, o);
    if (lane >= o) {
      off_t += a;
      off_r += b;
    }
  }
  const int tot_t = __shfl_sync(0xffffffffu, off_t, 7), tot_r = __shfl_sync(0xffffffffu, off_r, 7);
  off_t -= ntet_l;
  off_r -= ntri_l;
  for (int a = 0; a < ntet_l; ++a)
    for (int e = 0; e < 12; ++e) G.tet[off_t + a][e] = st[a][e];
  for (int a = 0; a < ntri_l; ++a)
    for (int e = 0; e < 12; ++e) G.tri[off_r + a][e] = tr[a][e];
  if (lane == 0) {
    G.n_tet = tot_t;
    G.n_tri = (sig != nullptr) ? tot_r : 0;
  }
  __syncthreads();
  double gacc[kGramPerLane], lacc[24], vol = 0.0;
#pragma unroll
  for (int t = 0; t < kGramPerLane; ++t) gacc[t] = 0.0;
#pragma unroll
  for (int e = 0; e < 24; ++e) lacc[e] = 0.0;
  double* pts = s_pt[warp];
  if (valid) {
    const double h = g.h, h3 = h * h * h, h2 = h * h;
    // stiffness: degree-5 rule, 32 points per round
    const int n_k = G.n_tet * kTet5Pts;
    for (int base = 0; base < n_k; base += 32) {
      const int it = base + lane;
      if (it < n_k) {
        const double* T = G.tet[it / kTet5Pts];
        const double* R = s_tet5 + (it % kTet5Pts) * 5;
        const double ux = T[3] - T[0], uy = T[4] - T[1], uz = T[5] - T[2];
        const double vx = T[6] - T[0], vy = T[7] - T[1], vz = T[8] - T[2];
        const double wx = T[9] - T[0], wy = T[10] - T[1], wz = T[11] - T[2];
        const double tv =
            fabs(ux * (vy * wz - vz * wy) - uy * (vx * wz - vz * wx) + uz * (vx * wy - vy * wx)) / 6.0;
        const double px = R[0] * T[0] + R[1] * T[3] + R[2] * T[6] + R[3] * T[9];
        const double py = R[0] * T[1] + R[1] * T[4] + R[2] * T[7] + R[3] * T[10];
        const double pz = R[0] * T[2] + R[1] * T[5] + R[2] * T[8] + R[3] * T[11];
        const double wq = R[4] * tv;
        double N[8], Gd[8][3];
        q1_shape_grad(px, py, pz, N, Gd);
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int d = 0; d < 3; ++d) pts[lane * 25 + 3 * a + d] = Gd[a][d];
        pts[lane * 25 + 24] = wq;
        vol += wq;
      }
      __syncwarp();
      const int np = min(32, n_k - base);
#pragma unroll
      for (int t = 0; t < kGramPerLane; ++t) {
        const int e = lane + 32 * t;
        if (e < kGram) {
          const int p = s_gp[e], q = s_gq[e];
          double a = 0.0;
          for (int k = 0; k < np; ++k) a += pts[k * 25 + 24] * pts[k * 25 + p] * pts[k * 25 + q];
          gacc[t] += a;
        }
      }
      __syncwarp();
    }
    // loads: body force (35-point rule) and boundary traction (facet rule)
    const int n_l = G.n_tet * kTetPts;
    const int n_all = n_l + G.n_tri * kTriPts;
    for (int it = lane; it < n_all; it += 32) {
      if (it < n_l) {
        const double* T = G.tet[it / kTetPts];
        const double* R = s_tet + (it % kTetPts) * 5;
        const double ux = T[3] - T[0], uy = T[4] - T[1], uz = T[5] - T[2];
        const double vx = T[6] - T[0], vy = T[7] - T[1], vz = T[8] - T[2];
        const double wx = T[9] - T[0], wy = T[10] - T[1], wz = T[11] - T[2];
        const double tv =
            fabs(ux * (vy * wz - vz * wy) - uy * (vx * wz - vz * wx) + uz * (vx * wy - vy * wx)) / 6.0;
        const double px = R[0] * T[0] + R[1] * T[3] + R[2] * T[6] + R[3] * T[9];
        const double py = R[0] * T[1] + R[1] * T[4] + R[2] * T[7] + R[3] * T[10];
        const double pz = R[0] * T[2] + R[1] * T[5] + R[2] * T[8] + R[3] * T[11];
        const double wq = R[4] * tv;
        double N[8];
        q1_shape(px, py, pz, N);
        double fh[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) fh[c] += N[a] * s_f[warp][a][c];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) lacc[3 * a + c] += wq * N[a] * fh[c] * h3;
      } else {
        const int r = it - n_l;
        const double* T = G.tri[r / kTriPts];
        const double* R = s_tri + (r % kTriPts) * 4;
        const double ux = T[3] - T[0], uy = T[4] - T[1], uz = T[5] - T[2];
        const double vx = T[6] - T[0], vy = T[7] - T[1], vz = T[8] - T[2];
        const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
        const double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
        const double px = R[0] * T[0] + R[1] * T[3] + R[2] * T[6];
        const double py = R[0] * T[1] + R[1] * T[4] + R[2] * T[7];
        const double pz = R[0] * T[2] + R[1] * T[5] + R[2] * T[8];
        const double wq = R[3] * area;
        double N[8];
        q1_shape(px, py, pz, N);
        double sh[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) sh[e] = 0.0;
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int e = 0; e < 9; ++e) sh[e] += N[a] * s_s[warp][a][e];
        double tq[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) tq[c] = sh[3 * c] * T[9] + sh[3 * c + 1] * T[10] + sh[3 * c + 2] * T[11];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) lacc[3 * a + c] += wq * N[a] * tq[c] * h2;
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 24; ++e) {
    double v = lacc[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    lacc[e] = v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vol += __shfl_xor_sync(0xffffffffu, vol, o);
  // Gm into shared memory (reusing the point buffer), then the element matrix
  __syncwarp();
#pragma unroll
  for (int t = 0; t < kGramPerLane; ++t) {
    const int e = lane + 32 * t;
    if (e < kGram) pts[e] = gacc[t];
  }
  __syncwarp();
  if (valid) {
    for (int e = lane; e < 576; e += 32) {
      const int p = e / 24, q = e % 24;
      const int a = p / 3, i = p % 3, b = q / 3, j = q % 3;
      double v = lam * pts[gram_index(p, q)] + mu * pts[gram_index(3 * a + j, 3 * b + i)];
      if (i == j)
        v += mu * (pts[gram_index(3 * a, 3 * b)] + pts[gram_index(3 * a + 1, 3 * b + 1)] +
                   pts[gram_index(3 * a + 2, 3 * b + 2)]);
      K_cut[kc * 576 + e] = v * g.h;
    }
    if (lane == 0) {
      for (int e = 0; e < 24; ++e) load_cut[kc * 24 + e] = lacc[e];
      eta[kc] = vol;
    }
  }
}

// elasticity right-hand side: b = sum_e load_e - A_FC g_C, three components per free node
__global__ void k_rhs_el(GridGeom g, int64_t n_dof, const int32_t* __restrict__ node_of_dof,
                         const int32_t* __restrict__ dof_of_node, const uint8_t* __restrict__ cell_type,
                         const int32_t* __restrict__ cut_index, const double* __restrict__ Kref,
                         const double* __restrict__ K_cut, const double* __restrict__ load_cut,
                         const double* __restrict__ kappa, const double* __restrict__ f,
                         const double* __restrict__ gval, const uint8_t* __restrict__ node_flags,
                         double* __restrict__ b) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof) return;
  const int64_t v = node_of_dof[d];
  const int i = (int)(v % (g.nx + 1)), j = (int)((v / (g.nx + 1)) % (g.ny + 1));
  const int k = (int)(v / ((int64_t)(g.nx + 1) * (g.ny + 1)));
  const double h = g.h, h3 = h * h * h;
  double sum[3] = {0.0, 0.0, 0.0};
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        const int ci = i + di, cj = j + dj, ck = k + dk;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx || cj >= g.ny || ck >= g.nz) continue;
        const int64_t c = g.cell(ci, cj, ck);
        const uint8_t t = cell_type[c];
        if (t == UFE_CELL_EXTERNAL) continue;
        const int a = (-di) + 2 * (-dj) + 4 * (-dk);
        const int32_t cx = t == UFE_CELL_CUT ? cut_index[c] : -1;
        for (int comp = 0; comp < 3; ++comp) {
          if (t == UFE_CELL_INTERNAL) {
            if (f) {
              double s = 0.0;
              for (int bb = 0; bb < 8; ++bb)
                s += q1_mhat(a, bb) * f[3 * g.node(ci + (bb & 1), cj + ((bb >> 1) & 1), ck + (bb >> 2)) + comp];
              sum[comp] += h3 * s;
            }
          } else {
            sum[comp] += load_cut[(int64_t)cx * 24 + 3 * a + comp];
          }
        }
        if (gval) {
          const double kap = kappa ? kappa[c] : 1.0;
          const double* Ke = t == UFE_CELL_INTERNAL ? Kref : K_cut + (int64_t)cx * 576;
          for (int bb = 0; bb < 8; ++bb) {
            const int64_t vb = g.node(ci + (bb & 1), cj + ((bb >> 1) & 1), ck + (bb >> 2));
            if (dof_of_node[vb] >= 0 || !(node_flags[vb] & 1)) continue;
            for (int comp = 0; comp < 3; ++comp)
              for (int jc = 0; jc < 3; ++jc)
                sum[comp] -= kap * Ke[(3 * a + comp) * 24 + 3 * bb + jc] * gval[3 * vb + jc];
          }
        }
      }
  for (int comp = 0; comp < 3; ++comp) b[3 * d + comp] = sum[comp];
}

void system_build_elastic(System& sys, const double* kappa, const double* f, const double* sig, const double* gval) {
  ensure_constants();
  Mesh& m = *sys.mesh;
  cudaStream_t s = sys.stream;
  const int64_t n_cut = m.n_cut;
  m.cut_cells.alloc(n_cut > 0 ? n_cut : 1, s);
  launch_cut_list(m, s);
  {
    std::vector<double> K(576);
    elastic_khat(sys.lam, sys.mu, K.data());
    for (double& x : K) x *= m.g.h;
    sys.Kref.alloc(576, s);
    UFE_CUDA(cudaMemcpyAsync(sys.Kref.p, K.data(), 576 * 8, cudaMemcpyHostToDevice, s));
    UFE_CUDA(cudaStreamSynchronize(s));
  }
  sys.K_cut.alloc((n_cut > 0 ? n_cut : 1) * 576, s);
  sys.load_cut.alloc((n_cut > 0 ? n_cut : 1) * 24, s);
  sys.eta.alloc(n_cut > 0 ? n_cut : 1, s);
  if (n_cut > 0) {
    TimedLaunch tl;
    tl.begin("integrate_cut", s);
    k_integrate_cut_el<<<grid_for(n_cut, kElWarps), kElWarps * 32, 0, s>>>(
        m.g, n_cut, m.cut_cells.p, m.phi.p, f, sig, sys.lam, sys.mu, sys.K_cut.p, sys.load_cut.p, sys.eta.p);
    UFE_CHECK_LAUNCH();
    tl.end(s);
  }
  sys.gnode.alloc(3 * m.g.n_nodes(), s);
  if (gval)
    UFE_CUDA(cudaMemcpyAsync(sys.gnode.p, gval, 3 * m.g.n_nodes() * 8, cudaMemcpyDeviceToDevice, s));
  else
    sys.gnode.zero();
  sys.b.alloc(3 * m.n_dof, s);
  k_rhs_el<<<grid_for(m.n_dof, 128), 128, 0, s>>>(m.g, m.n_dof, m.node_of_dof.p, m.dof_of_node.p, m.cell_type.p,
                                                   m.cut_index.p, sys.Kref.p, sys.K_cut.p, sys.load_cut.p, kappa, f,
                                                   gval, m.node_flags.p, sys.b.p);
  UFE_CHECK_LAUNCH();
}

}  // namespace ufe
