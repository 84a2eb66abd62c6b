"""Preconditioned conjugate gradients (oracle; test infrastructure only).

Sect. 5.1 stopping rule: stop once |r|_2 < tol |b|_2, with r the recursively
updated residual; the iteration count is the number of operator applications
to search directions.  Classical PCG takes beta = r_{k+1}.z_{k+1} / r_k.z_k;
the flexible form (Notay 2000, "Flexible conjugate gradients") takes
beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k, which tolerates a preconditioner that
varies from one application to the next (no counterpart in the paper).

Parity: pinned by termination in n steps on small SPD systems, by the exact
solve in one iteration when the preconditioner is A^-1, and by the Lanczos
relation between its alpha/beta and the spectrum of M A (tests).
"""
from __future__ import annotations

import numpy as np


class Breakdown(Exception):
    pass


def pcg(apply_A, b, apply_M, x0=None, rtol=1e-8, maxit=1000, flexible=False):
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0]
    alphas, betas = [], []
    it = 0
    converged = hist[0] < rtol
    if not converged:
        z = apply_M(r)
        p = z.copy()
        rz = r @ z
        while it < maxit:
            q = apply_A(p)
            pq = p @ q
            if not pq > 0:
                raise Breakdown(f"p.Ap = {pq} at iteration {it}")
            alpha = rz / pq
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            alphas.append(alpha)
            rn = np.linalg.norm(r)
            hist.append(rn / bnorm)
            if rn < rtol * bnorm:
                converged = True
                break
            z_new = apply_M(r)
            rz_new = r @ z_new
            beta = (r @ (z_new - z)) / rz if flexible else rz_new / rz
            betas.append(beta)
            p = z_new + beta * p
            z = z_new
            rz = rz_new
    true_res = np.linalg.norm(b - apply_A(x)) / bnorm if bnorm > 0 else 0.0
    return dict(x=x, iterations=it, converged=converged, history=np.array(hist),
                alphas=np.array(alphas), betas=np.array(betas), true_residual=true_res)


def lanczos_ritz(alphas, betas):
    """Ritz values of M A from the PCG coefficients (tridiagonal Lanczos matrix)."""
    m = len(alphas)
    T = np.zeros((m, m))
    for k in range(m):
        T[k, k] = 1.0 / alphas[k] + (betas[k - 1] / alphas[k - 1] if k > 0 else 0.0)
        if k + 1 < m:
            T[k, k + 1] = T[k + 1, k] = np.sqrt(betas[k]) / alphas[k]
    return np.linalg.eigvalsh(T)
