"""Plain FP64 CPU oracle for BDDC-preconditioned CG on unfitted Q1 elements.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import or run anything in this package.  The
product path (the CUDA library and its Python binding) never calls it and shares
no code, table or helper with it.

The oracle is written to be read against the paper (Badia & Verdugo,
"Robust and scalable domain decomposition solvers for unfitted finite element
methods"), not to be fast: numpy/scipy in float64, one obvious step at a time.

Modules and what they follow:
  * ``mesh``        -- cell classification, active set, DOFs, subdomain
                       aggregation, interface, neighbour sets (Sect. 2.1) and
                       geometric objects: standard (Sect. 3.2) and the first
                       variant of the improved coarse objects (Sect. 4.4);
  * ``quadrature``  -- Grundmann-Moeller simplex rules (published formula);
  * ``integration`` -- cut-cell integration by marching tetrahedra on the
                       Kuhn split of each cube, the bulk term of the element form
                       (Sect. 2.2) plus source and Neumann loads;
  * ``assembly``    -- element-by-element global operator and right-hand side
                       (Sect. 2.2), strong box Dirichlet and the pinned node (Sect. 5.1);
  * ``bddc``        -- sub-assembled local problems, coarse DOFs as object
                       means (Eq. coarse-dofs), topological weighting (Eq. weighting),
                       stiffness weighting (Eq. alge-weighting), harmonic extension,
                       and the preconditioner of Eq. bddc;
  * ``pcg``         -- (flexible) preconditioned CG with the relative residual
                       stopping rule of Sect. 5.1;
  * ``adjoint``     -- gradient of J = 1/2 |u - u_d|^2 w.r.t. per-cell
                       coefficients via the adjoint solve (no counterpart in the paper);
  * ``elasticity``  -- the vector-valued (Q1^3, isotropic linear elasticity)
                       variant of the same unfitted discretisation: 24x24 element
                       matrices, loads, assembly (no counterpart in the paper; the
                       BDDC of ``bddc`` takes 3 DOFs per node and rigid-mode
                       coarse rows for it);
  * ``multilevel``  -- three-level BDDC: the coarse problem of ``bddc`` itself
                       preconditioned by BDDC over groups of subdomains (Sect. 6
                       names multilevel BDDC as the way past one coarse
                       factorisation; the construction is reading R26).

Parity status per function is stated in each module header.
"""
