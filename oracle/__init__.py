"""CPU FP64 oracle for the PIE + MLFMA matrix-vector product (test infrastructure).

This package is test infrastructure, not product code.  Only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import it.  It shares no code with the CUDA library; the only inputs both
sides see come from ``pie_inputs`` (geometry and random numbers).

Contents, each module citing the passage of Guer & Erguel (2017) it follows:

* ``constants``  -- free-space constants (Section 2).
* ``quadrature`` -- triangle rules (Radon 7-point degree 5; collapsed Gauss).
* ``mesh``       -- RWG / pulse discretisation, N = T + E (Section 2).
* ``singular``   -- analytic potential integrals of 1/R and (r'-r)/R over a
  planar triangle, used for the near-singular Galerkin entries.
* ``moments``    -- per-triangle-pair moments of g (Section 2, after the
  integration by parts of Section 3).
* ``dense``      -- the dense Galerkin matrix Z of Eqs. (1)-(2) (Section 3,
  O(N^2) MOM).
* ``excitation`` -- plane-wave A^inc, Phi^inc and the right-hand side.
* ``farfield``   -- far-zone E from J and the RCS (Section 2).
* ``mie``        -- Mie series for a PEC sphere (Section 4 comparison).
* ``asd``        -- approximate stable diagonalization, Eqs. (4)-(5).
* ``tree``       -- cubic-box oct-tree and one-box-buffer lists (Section 3).
* ``mlfma``      -- aggregation / translation / disaggregation MVM (Section 3).
* ``gmres``      -- restarted GMRES (Section 4).
* ``levels``     -- the split of the product by the tree level that
  translates each pair (Section 3), for the per-level error of the far part.
* ``nearzone``   -- scattered field off the surface from J and the charge
  density (Section 2).
* ``search_asd`` -- the (tau, kappa a, N_theta) error search of Eqs. (4)-(5)
  (a report generator).

Parity status of each function is stated in its module header.
"""
