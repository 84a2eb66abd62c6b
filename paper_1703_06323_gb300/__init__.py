"""GB300 BDDC-PCG for unfitted (cut-cell) Q1 finite elements.

Badia & Verdugo, "Robust and scalable domain decomposition solvers for
unfitted finite element methods": PCG preconditioned by BDDC with stiffness
weighting and the improved (edge-splitting) coarse objects, on a Cartesian
background mesh whose cell blocks are the subdomains.

  * ``paper_1703_06323_gb300.ufe``       -- ctypes binding of the C ABI (include/ufe.h);
  * ``paper_1703_06323_gb300.solver``    -- a small Python convenience layer over it;
  * ``paper_1703_06323_gb300.inputs``    -- seeded synthetic problems;
  * ``paper_1703_06323_gb300.autograd``  -- torch.autograd wrapper of the adjoint gradient;
  * ``paper_1703_06323_gb300.build_ext`` -- builds libufe.so in-tree for sm_103a.

The binding is imported lazily so that the input generators work without the
CUDA library; the solver itself has no fallback and raises if the library is
missing.
"""
import importlib

__all__ = ["ufe", "solver", "inputs", "build_ext", "autograd"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
