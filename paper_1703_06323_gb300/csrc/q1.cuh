// Trilinear (Q1) shape functions on the unit cube and the closed-form unit-cube
// stiffness and mass matrices (vertex a has offsets (a & 1, (a >> 1) & 1, a >> 2)).
//   Khat_ab = sum_d k(a_d, b_d) prod_{d' != d} m(a_d', b_d'),  Mhat_ab = prod_d m(a_d, b_d),
//   k(same) = 1, k(diff) = -1, m(same) = 1/3, m(diff) = 1/6.
#pragma once

namespace ufe {

__host__ __device__ __forceinline__ double q1_khat(int a, int b) {
  double m[3], k[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const bool same = ((a >> d) & 1) == ((b >> d) & 1);
    m[d] = same ? (1.0 / 3.0) : (1.0 / 6.0);
    k[d] = same ? 1.0 : -1.0;
  }
  return k[0] * m[1] * m[2] + m[0] * k[1] * m[2] + m[0] * m[1] * k[2];
}

__host__ __device__ __forceinline__ double q1_mhat(int a, int b) {
  double r = 1.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) r *= (((a >> d) & 1) == ((b >> d) & 1)) ? (1.0 / 3.0) : (1.0 / 6.0);
  return r;
}

__device__ __forceinline__ void q1_shape(double x, double y, double z, double N[8]) {
  const double lx[2] = {1.0 - x, x}, ly[2] = {1.0 - y, y}, lz[2] = {1.0 - z, z};
#pragma unroll
  for (int a = 0; a < 8; ++a) N[a] = lx[a & 1] * ly[(a >> 1) & 1] * lz[a >> 2];
}

__device__ __forceinline__ void q1_shape_grad(double x, double y, double z, double N[8], double G[8][3]) {
  const double lx[2] = {1.0 - x, x}, ly[2] = {1.0 - y, y}, lz[2] = {1.0 - z, z};
  const double dl[2] = {-1.0, 1.0};
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
    N[a] = lx[ax] * ly[ay] * lz[az];
    G[a][0] = dl[ax] * ly[ay] * lz[az];
    G[a][1] = lx[ax] * dl[ay] * lz[az];
    G[a][2] = lx[ax] * ly[ay] * dl[az];
  }
}

}  // namespace ufe

namespace ufe {

// int over the unit cube of d_i N_a d_j N_b: a product of 1-D integrals of the
// linear shape functions n_0 = 1 - x, n_1 = x (slopes s_0 = -1, s_1 = +1):
//   int n_a' n_b' = s_a s_b,  int n_a' n_b = s_a / 2,  int n_a n_b = 1/3 (same) or 1/6
__host__ __device__ inline double q1_grad_grad(int a, int b, int i, int j) {
  double v = 1.0;
  for (int d = 0; d < 3; ++d) {
    const int ab = (a >> d) & 1, bb = (b >> d) & 1;
    const double sa = ab ? 1.0 : -1.0, sb = bb ? 1.0 : -1.0;
    const bool da = d == i, db = d == j;
    if (da && db)
      v *= sa * sb;
    else if (da)
      v *= 0.5 * sa;
    else if (db)
      v *= 0.5 * sb;
    else
      v *= ab == bb ? (1.0 / 3.0) : (1.0 / 6.0);
  }
  return v;
}

// unit-cube isotropic elasticity matrix (24 x 24, DOF 3 a + i):
//   K[3a+i][3b+j] = lambda G(a,i;b,j) + mu G(a,j;b,i) + delta_ij mu sum_d G(a,d;b,d),
//   G(a,i;b,j) = int d_i N_a d_j N_b
inline void elastic_khat(double lam, double mu, double* K) {
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      double lap = 0.0;
      for (int d = 0; d < 3; ++d) lap += q1_grad_grad(a, b, d, d);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double v = lam * q1_grad_grad(a, b, i, j) + mu * q1_grad_grad(a, b, j, i);
          if (i == j) v += mu * lap;
          K[(3 * a + i) * 24 + 3 * b + j] = v;
        }
    }
}

}  // namespace ufe
