"""CPU oracle for the hyper-reduced FE^2 online path (Lange, Huetter, Kiefer,
"A Monolithic Hyper ROM FE^2 Method with Clustered Training at Finite
Deformations", arXiv 2306.02687).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 NumPy/SciPy
restatement of the method, written from the paper's equations.  Only the test
suite, the smoke check and the benchmark's CPU-baseline leg may import it.  It
shares no code with the CUDA path (paper_2306_02687_gb300/) and never imports
it; the two meet only in the seeded generators of the `synthetic` module and in
ROM files written by `tests/golden/make_roms.py`.

Modules
  law       compressible Neo-Hooke law (stand-in constitutive law; the paper
            leaves the micro law open)
  polar     polar decomposition F = R U and its derivative (Sec. 3.2.2)
  rve       full-order periodic RVE finite elements (Sec. 2, Eqs. 4-8)
  rom       POD with elastic/inelastic split (Sec. 3.2.1), empirical cubature
            (Sec. 3.3, Box 1), ROM file writer
  reduced   hyper-reduced RVE evaluation with monolithic micro update, static
            condensation and rotation back (Sec. 3.2.2-3.2.3)
  macro     total-Lagrangian macro elements, monolithic and staggered Newton
            drivers (Sec. 2, Eq. 6; Sec. 3.2.3)
  adjoint   implicit-function adjoint of the converged reduced equilibrium
"""
