"""FP64 CPU oracle for the linear-finite-element compatibility-projection solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.
The product path (``paper_2105_03297_gb300``) never imports it, and this
package imports nothing from the product: the two share only the seeded input
generators in ``microstructures``.

Two independent formulations of the same discrete problem:

* ``fe_projection`` (O1): the paper's method written out plainly -- Fourier
  symbols of the linear-FE gradient stencils (Eq. genfourderiv), the
  small-strain projection G(k) = B (B^H B)^-1 B^H with G(0) = 0 (Eqs.
  discrete_projection_op, small-strain-eq2; the k = 0 rule of Sec. 2.3), the
  DFT pair of Appendix A (a direct matrix product per axis, or scipy's FFT), and a plain projected conjugate
  gradient (the gradient-based solver of Sec. 2.1).
* ``fem_assembly`` (O2): the conforming periodic linear-FE problem it is
  equivalent to (Sec. 2.6), assembled element by element in real space from
  the simplex shape functions and solved with a sparse direct solver.

``closed_forms`` holds the analytic pins (laminate moduli, Voigt/Reuss bounds,
the textbook small-strain Fourier projection, the literal index form of
Appendix B).

Every function works in float64.  Parity status of each function is stated
in its module header.
"""
