"""CPU oracle for inexact IETI-DP (Hofer, Langer, Takacs: "Inexact Dual-Primal
Isogeometric Tearing and Interconnecting Methods").

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never imports, links or runs it,
and this package never imports the product path.  The one module both sides
read is ``paper_1705_04531_gb300.workloads``, which only describes inputs.

Everything here is plain, slow FP64 numpy/scipy written from the paper:

* ``splines``   Cox-de Boor B-splines, tensor products, knot insertion (Sec. 2).
* ``geometry``  patch maps (identity grid, exact NURBS quarter annulus) and the
                model problem's right-hand sides (Eq. 1).
* ``assembly``  Galerkin stiffness / load / parameter mass per patch (Eq. 1,
                Sec. 3.2 for the parameter-domain mass).
* ``domain``    multipatch numbering, the conforming global system and its
                direct solve: the *definition* of the method's result.
* ``multigrid`` geometric h-multigrid with Gauss-Seidel smoothing (Sec. 4).
* ``ietidp``    tearing, jump operator, primal constraints, energy-minimizing
                primal basis (Eq. 6), local Neumann solves (Eq. 7), scaled
                Dirichlet preconditioner and the dual PCG for Eq. 4, in the
                D-D (direct), D-MG and MG-MG (multigrid) variants of Sec. 3.3.
* ``saddle``    MG-MG-S: Bramble-Pasciak CG on the saddle-point system Eq. 2.
* ``szcg``      the primal basis by Schoeberl-Zulehner preconditioned CG
                (Sec. 3.2).
* ``sharded``   the dual PCG with its patches sharded over ranks (the
                exchange step of a multi-GPU solve: all-reduce of r_Pi and of
                the partial jump-operator outputs).

Parity status of each function is stated in its module header.
"""
