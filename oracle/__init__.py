"""FP64 CPU oracle for the energy-conserving DG discretisation of the
time-domain Maxwell equations (Koutschan, Lehrenfeld, Schoeberl,
"Computer Algebra meets Finite Elements", arXiv:1104.4208).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
does, and this package imports nothing from the product.

What it computes is the plain definition of the method:
  * the Dubiner basis of Sec. 4.2.2 (3D) and Eq. (4) (faces), evaluated by
    the textbook Jacobi three-term recurrence with forward-mode gradients;
  * element and facet integrals of the weak form of Sec. 2.1 (stabilized
    central flux, Sec. 2.1 final system) by brute-force Gauss quadrature in
    PHYSICAL space: covariant basis functions F^{-T} phi(Phi^{-1} x), physical
    curls by the chain rule, physical outward normals, neighbour fields
    evaluated at the same physical point through the neighbour's own inverse
    map -- no reference-element identities, no recurrences, no face frames;
  * block mass matrices assembled by quadrature and inverted by Cholesky;
  * symplectic Euler / leapfrog of Sec. 3 and the discrete energy of Sec. 2.1;
  * the same scheme for 2D TE fields on triangles (``dg2d``: E in the plane,
    H along z, the Eq. (4) basis), the oracle of a 2D triangle solver;
  * material parameters varying inside flat elements (``varcoef``) and curved
    elements from a smooth global map (``curved``): the exact mass and the
    approximate inverse mass of Sec. 3.3.2.

Readings of the paper taken here (the same as the CUDA path's):
  * p is the degree of E; H has degree p-1 (Sec. 2, spaces V^{k+1}, V^k).
  * The facet terms carry the sign that makes the scheme consistent with the
    integration-by-parts identity (curl u, v)_T = (u, curl v)_T + (nu x u, v)_dT
    for the outward normal nu:  r_E(e) = (H, curl e)_T - ({{H}} x nu, e)_dT and
    r_H(h) = -(curl E, h)_T - (1/2 [[E]] x nu, h)_dT.  The printed formulas
    carry the opposite sign on both facet terms (equivalent to an inward
    normal); both choices are skew, only this one is consistent.
  * H^F evolves by (h_F/alpha) (dH^F/dt, h^F)_F = ([[E]] x nu_F, h^F)_F, so that
    eliminating H^F reproduces the stabilisation S(E,e) with weight alpha/h
    and H^F = alpha [[E]] x nu / (i w h) as defined in Sec. 2.1;
    alpha = alpha0 p^2, h_F = min over the adjacent tets of 3|T|/|F|.
  * PEC boundary faces use the ghost state E_ext = -E, H_ext = H.
"""
