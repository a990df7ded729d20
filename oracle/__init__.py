"""CPU FP64 oracle for the IgA + p-multigrid + MGRIT heat solver (arXiv 2107.05337).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline legs of ``bench.py`` may import it.  It shares no code with
the CUDA path in ``paper_2107_05337_gb300`` (no kernels, headers, helpers,
tables or constant generators); the only module both sides use is the seeded
input generator ``paper_2107_05337_gb300.inputs``, which holds none of the
method's arithmetic.

Everything here is plain NumPy / SciPy in float64, written for a reader who
checks it against the paper by eye:

* ``bspline``   -- open knot vectors and the Cox--de Boor recursion (Sec. 2).
* ``geometry``  -- the parametric maps F: (0,1)^2 -> Omega (Sec. 2).
* ``assembly``  -- Gauss-quadrature mass/stiffness/transfer matrices, load
  vectors, L2 projection, Dirichlet elimination (Sec. 2, Eq. (PM) of Sec. 4).
* ``timestep``  -- sequential backward Euler with a sparse direct solve
  (Sec. 3, block forward solve of the space-time system).
* ``mgrit``     -- two-level / multilevel MGRIT with FCF relaxation,
  injection and ideal interpolation (Sec. 3, the MGRIT algorithm box).
* ``pmg``       -- p-multigrid: ILUT smoother, L2-projection transfers with
  lumped masses, h-multigrid W-cycle at p=1 with Gauss--Seidel and a direct
  coarsest solve (Sec. 4, steps 1-5 and Fig. 5).

Parity status of each function is recorded in its module header; every
function here is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""
