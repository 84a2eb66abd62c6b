"""Weak Dirichlet conditions on the unfitted boundary by Nitsche's method (oracle; test
infrastructure only).

Sect. 2.2: on every cut cell e whose part of the boundary carries Dirichlet data g^D,
the bilinear form gains
    int_{Gamma_D cap e} ( beta_e u v - v (n . grad u) - u (n . grad v) ) dS
and the right-hand side
    int_{Gamma_D cap e} ( beta_e v g^D - (n . grad v) g^D ) dS,
with n the outward normal of Omega.  Coercivity holds for beta_e >= C_e, the largest
eigenvalue of the generalised eigenproblem B_e x = lambda D_e x with
    D_e(u, v) = int_{e cap Omega} grad u . grad v,
    B_e(u, v) = int_{Gamma_D cap e} (n . grad u)(n . grad v) dS
(both vanish on the constants, so the problem lives on their complement); the paper
takes beta_e = 2 C_e (Eq. local-eigenvals).

Readings (the paper leaves them open):
  * the Dirichlet boundary inside a cut cell is the same tet-linear surface that the
    Neumann data use (marching tetrahedra, Sect. 2.2 integration cells), its normal the
    gradient of the tet-linear level set;
  * g^D is the Q1 interpolant of nodal values (the problem's Dirichlet values);
  * C_e is computed on the complement of the constants after a symmetric Jacobi
    scaling by diag(D_e)^-1/2 (a congruence: the eigenvalues do not change), in an
    orthonormal (Householder) basis of that complement, by a Cholesky reduction and a
    symmetric eigensolver.

Parity: pinned (tests/test_oracle_nitsche.py) by C_e against the nonzero spectrum of
pinv(D_e) B_e and Rayleigh quotients of random vectors, the constants in the kernel of
both forms, the per-cell coercivity bound A_e - D_e / 2 >= 0 that beta_e = 2 C_e
guarantees, the exact reproduction of a linear solution with weak Dirichlet data on a
plane cut (consistency of the Nitsche form), and second-order convergence of the
manufactured solution on a sphere with weak Dirichlet data.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .quadrature import TRI_BARY, TRI_W


def _q1_shape(xi):
    from .integration import q1_shape
    return q1_shape(xi)


def _q1_grad(xi):
    from .integration import q1_grad
    return q1_grad(xi)


def facet_forms(tris_normals):
    """Unit-cube facet forms of one cut cell from its boundary triangles.

    tris_normals: list of (triangle (3,3), unit normal (3,)) in unit-cube coordinates.
    Returns (M, C, B) (8x8 each): M_ab = int N_a N_b dS, C_ab = int N_a (n . grad N_b) dS,
    B_ab = int (n . grad N_a)(n . grad N_b) dS over the triangles."""
    M = np.zeros((8, 8))
    C = np.zeros((8, 8))
    B = np.zeros((8, 8))
    for T, normal in tris_normals:
        area = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
        if area == 0.0:
            continue
        xq = TRI_BARY @ T
        wq = TRI_W * area
        N = _q1_shape(xq)                     # (m, 8)
        dn = _q1_grad(xq) @ normal            # (m, 8): n . grad N_a
        M += np.einsum("q,qa,qb->ab", wq, N, N)
        C += np.einsum("q,qa,qb->ab", wq, N, dn)
        B += np.einsum("q,qa,qb->ab", wq, dn, dn)
    return M, C, B


def _householder_complement(k):
    """Orthonormal basis (8 x 7) of the complement of the vector k."""
    k = k / np.linalg.norm(k)
    e = np.zeros_like(k)
    e[0] = 1.0
    v = k + np.copysign(1.0, k[0]) * e
    H = np.eye(k.size) - 2.0 * np.outer(v, v) / (v @ v)
    return H[:, 1:]                           # H e_0 = -sign(k_0) k; the other columns span k^perp


def nitsche_constant(D, B):
    """C_e = largest eigenvalue of B x = lambda D x on the complement of the constants."""
    s = 1.0 / np.sqrt(np.diag(D))
    Ds = D * np.outer(s, s)
    Bs = B * np.outer(s, s)
    V = _householder_complement(1.0 / s)      # kernel of the scaled D: S^-1 (1, ..., 1)
    D7 = V.T @ Ds @ V
    B7 = V.T @ Bs @ V
    L = np.linalg.cholesky(0.5 * (D7 + D7.T))
    Li = sla.solve_triangular(L, np.eye(7), lower=True)
    G = Li @ B7 @ Li.T
    return float(np.linalg.eigvalsh(0.5 * (G + G.T))[-1])


def nitsche_cell(K_unit, tris_normals, g8, h):
    """Nitsche terms of one cut cell in physical units.

    K_unit: int_{e cap Omega} grad N_a . grad N_b in unit-cube coordinates (8x8);
    tris_normals: its boundary triangles; g8: nodal Dirichlet data; h: cell size.
    Returns (Nmat (8x8), load (8,), beta) with beta = 2 C_e; Nmat and load are added to
    the cell's stiffness matrix and load vector."""
    M, C, B = facet_forms(tris_normals)
    if not np.any(B):
        return np.zeros((8, 8)), np.zeros(8), 0.0
    lam = nitsche_constant(K_unit, B)         # unit-cube C_e; physical C_e = lam / h
    beta_unit = 2.0 * lam
    Nmat = h * (beta_unit * M - C - C.T)
    load = h * (beta_unit * (M @ g8) - C.T @ g8)
    return Nmat, load, beta_unit / h
