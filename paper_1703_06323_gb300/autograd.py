"""torch.autograd wrapper: per-cell coefficient -> solution, with an adjoint backward.

forward(kappa)  assembles A(kappa) = sum_e kappa_e Khat_e on the device, sets up BDDC
                and solves A u = b with PCG (ufe_mesh_create / ufe_assemble /
                ufe_bddc_setup / ufe_pcg_solve);
backward(g_u)   solves A lambda = g_u with the same BDDC-PCG (A is symmetric) and
                contracts dJ/dkappa_e = -ubar_e^T Khat_e lambda_e in one kernel
                (ufe_adjoint).  No counterpart in the paper.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ufe
from .solver import Solver


def _dev(a, device):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.float64).contiguous()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)


class PoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, problem, options):
        opts = dict(options or {})
        rtol = opts.pop("rtol", 1e-8)
        maxit = opts.pop("maxit", 1000)
        dev = kappa.device
        arrays = {"phi": _dev(problem.phi, dev), "f": _dev(problem.f, dev), "q": _dev(problem.q, dev),
                  "g": _dev(problem.dirichlet_values, dev), "kappa": kappa.detach().contiguous()}
        solver = Solver(problem, arrays=arrays, **opts)
        x = torch.zeros(solver.n_dof, dtype=torch.float64, device=dev)
        solver.solve(x0=x, rtol=rtol, maxit=maxit)
        ctx.solver = solver
        ctx.rtol, ctx.maxit = rtol, maxit
        ctx.n_cells = kappa.numel()
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        S = ctx.solver
        lam = torch.zeros_like(x)
        g = torch.empty(ctx.n_cells, dtype=torch.float64, device=x.device)
        try:
            ufe.ufe_adjoint(S.system, S.bddc, x, grad_x.contiguous(), lam, g, rtol=ctx.rtol, maxit=ctx.maxit)
        finally:
            S.close()
        return g, None, None


def solve(kappa, problem, **options):
    """u(kappa) for one problem; differentiable with respect to kappa."""
    return PoissonSolve.apply(kappa, problem, options)


def lumped_mass(problem, device):
    """m_xi = int_Omega phi_xi per free DOF (the right-hand side of f = 1 without data)."""
    mesh = ufe.ufe_mesh_create(problem.box_lo, problem.box_hi, problem.cells, problem.sub_cells,
                               _dev(problem.phi, device), problem.dirichlet_face_mask, problem.pin_node)
    try:
        n = ufe.ufe_mesh_get_info(mesh)["n_dof"]
        one = torch.ones(problem.n_nodes, dtype=torch.float64, device=device)
        sysh = ufe.ufe_assemble(mesh, None, one, None, None)
        try:
            return torch.from_numpy(ufe.ufe_system_get_rhs(sysh, n)).to(device)
        finally:
            ufe.ufe_system_destroy(sysh)
    finally:
        ufe.ufe_mesh_destroy(mesh)
