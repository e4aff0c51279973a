"""FP64 CPU oracle for the surface-conductive-absorber PMCHW operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference leg may use it.  It shares no code with the CUDA path;
the two meet only in the seeded input generators of ``synth``.

It is written for readability, in numpy float64 / complex128, and follows the
paper (Zhang et al., "A Novel Boundary Element Method Using Surface Conductive
Absorbers for Full-Wave Analysis of 3-D Nanophotonics"):

* ``mesh``       RWG basis on a closed triangle mesh, L/R edge classes and the
                 unknown vector x = [J^L, M^L, J_e^R, J_i^R, M^R] (Appendix A).
* ``integrals``  potential integrals over flat triangles (singularity
                 extraction with the closed-form 1/R and grad(1/R) integrals).
* ``operator``   O1: the Galerkin PMCHW operator with the absorber rows
                 (Eqs. 1-3, 13, 14 with the MPIE operators of Eqs. 15-16),
                 direct matrix-free matvec, dense assembly and LU solve.
* ``pfft``       O2: the plain definition of the grid-accelerated operator:
                 explicit Lagrange projection / interpolation matrices, a
                 zero-padded grid convolution with G(0)=0, and the explicit
                 near-field precorrection.
* ``excitation`` incident fields (plane wave, dipole, complex-source beam) and
                 the tested right-hand side b (Appendix A).
* ``sigma``      conductivity profiles (the monomial of Eq. 23, and a cubic
                 B-spline by the Cox-de Boor recursion).
* ``post``       SWR -> r, fields at points, on-axis reflection fit, the
                 decay-rate fit of Sec. III, far field.
* ``toeplitz``   the exact block-Toeplitz product of O1 on a straight extruded
                 guide (Appendix B), by circulant embedding along the slices.
* ``mie``        Mie series for a dielectric sphere, optionally with a surface
                 conductivity sheet (textbook, derived from the boundary
                 conditions of Eq. 4).

Units: lengths in um; fields normalised so that the free-space impedance is 1
(J is stored as eta0*J, H as eta0*H, sigma as eta0*sigma).  This is a diagonal
rescaling of the paper's system that makes all blocks of A comparable.
"""

ETA0 = 376.730313668  # free-space impedance [ohm], CODATA 2018
