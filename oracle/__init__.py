"""Plain, slow FP64 CPU oracle of the MS-GFEM local stage (arXiv 2211.13893).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or execute anything in this
package.  The GPU product path (``paper_2211_13893_gb300``) never imports it,
and this package imports nothing from the product path: the two share only the
seeded input generators in ``workloads/``.

Each function follows the paper's definitions step by step, with library
primitives (sparse LU, dense Cholesky, symmetric eigensolvers) as steps:

* ``material``  orthotropic ply tensor and its rotation (Sec. 2, Eq. eq-hooke;
  Sec. 5.1 "standard tensor rotations").
* ``element``   trilinear hexahedron stiffness by 2x2x2 Gauss quadrature
  (Eq. weak_form, Eq. element_stiffness).
* ``mesh``      structured laminated-beam mesh, clamped x = 0 face, traction
  load on x = L (Eq. weak_form, b(v)); ``HexMesh`` for structured meshes with
  given node coordinates and per-element ply frames (the curved C-section).
* ``assemble``  global and subdomain-restricted stiffness (Eqs.
  element_stiffness, restricted_bilinear_form).
* ``partition`` non-overlapping boxes, overlap and oversampling layers, the DoF
  classes B1/B2/B3 (Sec. 4.3) and the partition of unity (Sec. 4.2).
* ``local``     the A-harmonic local eigenproblem (Eq.
  AHarmonicGeneralizeEigenProblem, Eq. algebraicAharmonic) solved densely in
  reduced form, and the local particular function (Eq. up_r).
* ``arpack``    the paper's own solver design: shift-invert Lanczos (ARPACK) on
  the saddle-point pencil with a sparse LU (Sec. 4.5).
* ``coarse``    PoU-weighted basis with Gram-Schmidt (Sec. 4.3-4.4), the coarse
  Galerkin problem (Eq. GFEM_coarse_approximation) and the energy error; local
  basis sizes from n_loc or from the eigenvalue threshold (Sec. 5.5).
* ``fine``      the fine-scale FE solution u_h (Eq. fe_matrix_system) by a
  direct sparse solve.
* ``errors``    the relative L2 errors e_d and e_eps of the displacement and
  strain fields (Sec. 5.4).
* ``geneo``     the GenEO local eigenproblem and coarse space, the paper's
  comparison method (Sec. 2.3, Eq. bilinearGeneralizeEigenProblem).
* ``schwarz``   two-level additive Schwarz preconditioned CG, the fine-scale
  solver a coarse space preconditions (Sec. 2.3, Sec. 5.4).

Parity pins live in ``tests/test_oracle_*.py``.
"""
