"""Plain FP64 CPU oracle for the CALCLENS lens-plane hot path (Becker 2012).

TEST INFRASTRUCTURE ONLY.  This package restates the paper's method slowly and
plainly so that the CUDA path can be checked against it.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import it.  It shares no code, tables or constants with the
CUDA library (``paper_1210_3069_gb300``) and never imports it.

Modules (each function cites the passage of the paper it follows):

* ``healpix``  - HEALPix RING/NEST geometry from Gorski et al. (2005), the
  pixelisation the paper uses for rays, bundles and the SHT grid (Sec. 3,
  Sec. 3.1).
* ``binning``  - particle deposit to pixel counts and the plane source
  kappa^(m) (Sec. 3.2, Eq. lenspoisson).
* ``sht``      - spherical-harmonic analysis / synthesis on HEALPix rings,
  the harmonic Poisson solve psi_lm = -kappa_lm / l(l+1) and the derivative
  synthesis of the pure-SHT solver (Sec. 3.2).
* ``interp``   - HEALPix ring-bilinear interpolation (Sec. 3.2, Sec. 3.3).
* ``mg``       - the FAS multigrid patch solver of the SHT+MG method
  (Sec. 3.2) and its fourth-order finite-difference derivatives.
* ``geometry`` - sphere differential geometry of Appendix A: deflection and
  shear from potential derivatives, tangent bases and their rotations.
* ``rays``     - multiple-plane ray recursion (Eq. betaprop, Eq. posprop,
  Eq. Atraj), parallel transport (Appendix B) and the radial interpolation
  to galaxies (Appendix D, Eq. gatraj).
* ``spectra``  - convergence, E/B-mode shear and rotation power spectra
  (Sec. 5).

Floating point is IEEE FP64 throughout; elementwise torch ops on CPU round
each operation separately (no fused multiply-add), which is what makes the
integer pixel indices reproducible bit for bit.
"""
