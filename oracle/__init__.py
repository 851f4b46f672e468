"""Plain, slow FP64 CPU oracle for the quasi-matrix-free hybrid multigrid hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path; the only common module is ``synthetic`` (seeded
input fields, no method arithmetic).

Every function follows a passage of Weinzierl & Weinzierl, "Quasi-matrix-free
hybrid multigrid on dynamically adaptive Cartesian grids" (arXiv:1607.00648),
cited by section, equation, algorithm or appendix:

* ``spacetree``  -- k=3 spacetree, vertex classes, Peano order, level tables (Sect. 3, App. A)
* ``fem``        -- d-linear FEM element matrices and level operators (Sect. 4, eq. "03_solver:stencils")
* ``boxmg``      -- BoxMG prolongation via one C(s) p = f solve per patch corner (Sect. 4.4, App. C)
* ``galerkin``   -- Galerkin coarse operators A_{l-1} = R A_l P and hierarchical deltas (Sect. 4.3, Sect. 5)
* ``multigrid``  -- damped Jacobi and block Jacobi smoothing, residual, transfers, V-cycle, solve,
                    additive traversal (Sect. 4.1, 4.2, Alg. 1, Alg. 2)
* ``codec``      -- the BF16/FP16 + per-vertex FP32 scale storage of the deltas (Sect. 5, as a dtype)
* ``bpa``        -- the paper's own byte codec of the deltas, f_bpa = m 2^e with a per-operator bpa (Sect. 5)
"""
