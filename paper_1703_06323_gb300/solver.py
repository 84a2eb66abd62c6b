"""Convenience layer: one Problem -> mesh, system, preconditioner, solve.

Each step is one C-ABI call (see include/ufe.h); this module only keeps the
handles together and frees them in the right order.
"""
from __future__ import annotations

import numpy as np

from . import ufe

WEIGHTING = {"stiffness": ufe.WEIGHT_STIFFNESS, "topological": ufe.WEIGHT_TOPOLOGICAL}
OBJECTS = {"std": ufe.OBJECTS_STANDARD, "v1": ufe.OBJECTS_VARIANT1, "v2": ufe.OBJECTS_VARIANT2}
COARSE = {"c": ufe.COARSE_C, "ce": ufe.COARSE_CE, "cef": ufe.COARSE_CEF}
PRECISION = {"fp64": ufe.PREC_FP64, "mixed": ufe.PREC_MIXED}
COARSE_SOLVER = {"auto": ufe.COARSE_SOLVER_AUTO, "dense": ufe.COARSE_SOLVER_DENSE, "cr": ufe.COARSE_SOLVER_CR,
                 "bddc": ufe.COARSE_SOLVER_BDDC}


class Solver:
    """Owns the ufe handles of one problem (host numpy inputs or torch CUDA tensors)."""

    def __init__(self, problem, weighting="stiffness", objects="v1", coarse="cef", precision="fp64", stream=None,
                 arrays=None, coarse_solver="auto", coarse_group=0, coarse_keep_corners=False):
        p = problem
        a = arrays or {}
        self.mesh = ufe.ufe_mesh_create(p.box_lo, p.box_hi, p.cells, p.sub_cells, a.get("phi", p.phi),
                                        p.dirichlet_face_mask, p.pin_node, stream=stream)
        self.system = None
        self.bddc = None
        try:
            self.info = ufe.ufe_mesh_get_info(self.mesh)
            if getattr(p, "ncomp", 1) == 3:
                E, nu = p.lame
                self.system = ufe.ufe_assemble_elastic(self.mesh, E, nu, a.get("kappa", p.kappa), a.get("f", p.f),
                                                       a.get("q", p.q), a.get("g", p.dirichlet_values))
            elif getattr(p, "weak_dirichlet", False):
                self.system = ufe.ufe_assemble_nitsche(self.mesh, a.get("f", p.f), a.get("g", p.dirichlet_values))
            else:
                self.system = ufe.ufe_assemble(self.mesh, a.get("kappa", p.kappa), a.get("f", p.f),
                                               a.get("q", p.q), a.get("g", p.dirichlet_values))
            self.bddc = ufe.ufe_bddc_setup(self.system, WEIGHTING[weighting], OBJECTS[objects], COARSE[coarse],
                                           PRECISION[precision], COARSE_SOLVER[coarse_solver], coarse_group,
                                           int(bool(coarse_keep_corners)))
            self.bddc_info = ufe.ufe_bddc_get_info(self.bddc)
        except Exception:
            self.close()
            raise
        # length of solution vectors: ncomp * free nodes (3 per node for elasticity)
        self.ncomp = ufe.ufe_system_get_info(self.system)["ncomp"]
        self.n_dof = ufe.ufe_system_get_info(self.system)["n"]

    def rhs(self):
        return ufe.ufe_system_get_rhs(self.system, self.n_dof)

    def apply(self, x):
        return ufe.ufe_system_apply(self.system, x)

    def precondition(self, r):
        return ufe.ufe_bddc_apply(self.bddc, r)

    def solve(self, b=None, x0=None, rtol=1e-8, maxit=1000, flexible=-1, check_every=8, raise_on_error=True):
        x = np.zeros(self.n_dof) if x0 is None else x0
        st, info = ufe.ufe_pcg_solve(self.system, self.bddc, b, x, rtol=rtol, maxit=maxit, flexible=flexible,
                                     check_every=check_every, raise_on_error=raise_on_error)
        info["status"] = st
        return x, info

    def close(self):
        if self.bddc is not None:
            ufe.ufe_bddc_destroy(self.bddc)
            self.bddc = None
        if self.system is not None:
            ufe.ufe_system_destroy(self.system)
            self.system = None
        if self.mesh is not None:
            ufe.ufe_mesh_destroy(self.mesh)
            self.mesh = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
