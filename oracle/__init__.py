"""FP64 CPU oracle for the stabilised Q1-Q1 natural-convection solver.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path (the
CUDA library and its Python binding) never imports it, and this package never
imports the product path.

It is the plain definition of what the GPU path computes, for the paper
"Large scale three-dimensional topology optimisation of heat sinks cooled by
natural convection" (Alexandersen, Sigmund, Aage):

* ``grid``      structured hex grid, node/element numbering, boundary conditions
* ``element``   element residual of the stabilised weak form (Sec. 2, Sec. 4, App. B)
* ``assemble``  global residual, complex-step element Jacobians assembled to CSR
* ``solve``     damped Newton with the polynomial line search (Sec. 5.1), direct
                linear solves, objective, adjoint and design sensitivities (Sec. 3.2),
                the Gram-Schmidt step of the FGMRES Arnoldi process (Sec. 5.2)
* ``filter``    the PDE density filter (Sec. 3.2)
* ``mma``       the method of moving asymptotes for the volume-constrained
                problem of Sec. 3.2 (one constraint, dual solved by bisection)
* ``multigrid`` the trilinear prolongation and the Galerkin coarse operator
                P^T A P of the multigrid preconditioner (Sec. 5.2)

Everything is NumPy/SciPy in float64 (complex128 for the complex-step
derivatives). Nothing is blocked, fused or reordered beyond the definitions.

Parity status: the weak form itself is a reading (the paper defers it to its
reference [Alexandersen2014]); it is pinned by invariants (hydrostatic rest,
pure conduction, slab solutions, manufactured-solution convergence, FD of the
Jacobian and of the sensitivities, printed tau derivatives), not by printed
values. Paper-level objective values (Table 5) are parity unpinned: they need
the paper's optimised designs.
"""
