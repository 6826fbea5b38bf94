"""Plain, slow, FP64 CPU oracle of the hybridized implicit-explicit FR stage.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the product
path (the CUDA library and its Python binding) never does.

Each module restates one part of Pereira & Vermeire, *Hybridized
Implicit-Explicit Flux Reconstruction Methods* (arXiv 2401.16632), citing the
section / equation it follows:

* ``basis``     -- Gauss-Legendre solution points, Lagrange basis, Radau
                   (DG-recovering) correction functions (Sec. 2, eqs. frsolution,
                   frfluxd, fluxcorrection, dsklnf).
* ``geometry``  -- bilinear element mapping, Jacobian, adjugate metrics and face
                   normals (Sec. 2, eqs. d9sfxda, 3289u4, 8923i).
* ``physics``   -- advection-diffusion and compressible Navier-Stokes fluxes,
                   written so they also accept complex arguments (complex-step
                   differentiation).
* ``fr``        -- the FR residual (eq. freq1), the hybridized residual with the
                   trace variable (eqs. hfrriemann, hfr1) and the transmission
                   conditions / trace residual (eqs. 5treerf, 53904jn, hfr2,
                   hfrimex).
* ``blocks``    -- element Jacobian blocks A, B, C, D (eqs. elemA, elemsystem,
                   elemsystemB) by complex-step differentiation of the element
                   residual, and the monolithic global Jacobian.
* ``solve``     -- static condensation, assembly, GMRES and back-substitution
                   (Sec. 3.2, eqs. assembly, assembly2, localproblems).
* ``boundary``  -- boundary faces: hybridized no-slip adiabatic walls and far field (eq. hfr2's
                   boundary term), FR ghost state on explicit far-field faces.
* ``efr``       -- interior-embedded FR (Sec. 2.2): the trace continuous on the implicit
                   skeleton at GLL face points, its transmission conditions, and the
                   condensed and monolithic Newton steps.
* ``fr3d``      -- the FR / HFR residual, blocks and condensed / monolithic Newton steps on
                   hexahedra (trilinear map, six faces of (p+1)^2 points; Sec. 5.3's 3D
                   cases), with ``physics.NavierStokes3D``.
* ``fr_mixed``  -- the FR / HFR residual and trace residual on meshes whose elements
                   carry different degrees (Sec. 3.2, p-adaptive meshes): face points
                   of the higher degree, L2 projection of face jumps back to each side.
* ``blocks_mixed`` -- element blocks of uneven shapes on such meshes and the condensed
                   Newton step, checked against the monolithic step.
* ``stepping``  -- Newton on the DIRK stage equations (eqs. 9oind, 23nffsd), the
                   SDIRK2 and IMEX tableaux (Table butcherimex) and the IMEX step
                   (Algorithm 1, eqs. explicitimex, hfrimex).

Readings of points the paper leaves open are listed in the module docstrings
where they are used.
"""
