"""Plain, slow FP64 CPU oracle for the Stokes layer-operator apply on SH drop surfaces.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package: only the
tests, the smoke check and the CPU-baseline leg of the benchmark use it.  It shares no code
with the CUDA library (no kernels, tables, constants or helpers); both sides consume the
same seeded inputs.

Modules, each following the passage of Sorgentone & Tornberg (arXiv 1707.02156) it cites:
  sh        grid, normalised Legendre functions, analysis/synthesis, derivatives (Sec. 1.1, 2.1, App. A)
  wigner    Wigner small-d matrices and coefficient rotation (App. B)
  geometry  fundamental forms, normal, curvature, interfacial force (Table 2, Sec. 1)
  layer     singular self quadrature (Thm 1, Sec. 2.2), regular and upsampled pair sums and the
            region split (Sec. 2.3), near-singular interpolation (Sec. 2.3), Galerkin projection (Sec. 1.2)
  gmres     restarted GMRES with modified Gram-Schmidt (Sec. 6)
  timestep  midpoint step of the drop shapes with the surfactant held fixed (Sec. 3, Alg. 1)
  surfactant  surface gradient, divergence and Laplacian; the transport terms of Eq. surfactant0;
            IMEX-2 and IMEX-1 steps with the preconditioned implicit solve; the coupled
            drop/surfactant step and the adaptive step size of Alg. 1 (Sec. 3)
  reparam   angle reparametrisation with the adaptive cutoff (Sec. 4, Alg. 2)
  brute     adaptive polar quadrature used only as a reference: the singular self-integral and
            integrals at points just off the surface

The near-singular (Omega_2) interpolation on deformed shapes has no closed form; it is pinned by
its convergence, as the degree grows, to the brute-force integral at points just off the surface.
"""
