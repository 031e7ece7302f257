"""CPU FP64 oracle for the FFT-based diffuse-scattering calculation of arXiv 1809.07088.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test-suite (tests/), the smoke check of
__graft_entry__ and the CPU-baseline / reference legs of bench.py may import, call, link or
execute anything under oracle/.  The product path (paper_1809_07088_gb300) never does, and it
shares no code, table or constant generator with this package: the only thing both sides read
is the seeded input models of the separate `synthetic` module.

Contents, each function citing the passage it follows:
  core.structure_factor ........ Eq. sf, by a plain loop in C (direct.c), FP64
  core.*_intensity_direct ...... Eqs. intensity_sf, bragg_diffuse_sf, bragg_sf, bragg_sf_disp,
                                 mag_sf, mag_intensity, mag_projection (direct sum, "part 1")
  core.*_intensity_fft ......... Section III: Eqs. fft, comp_ft, comp_sf_diffuse,
                                 total_sf_taylor, U_fft, A_fft, mag_ft (the method, "part 2");
                                 numpy's FFT is the library step
  core.monomials, taylor_order, x_max, truncation_bound ..... Section III C
  core.zone_taylor_orders ...... the Section III C bound applied per zone H (|Q.u| <= |Q||u|)
  noise.subbox_intensity ....... Section V A, every lattice point an origin, brute force
  noise.lanczos_resample ....... Section V B, Eqs. intensity_convol_finite, weight_sinc,
                                 windowed_sinc, lanczos, and the 1/m' variant
  adjoint.*_chi2_grad .......... chain rule of Eq. sf for chi^2 (no counterpart in the paper)

Pins (tests/test_oracle_*.py, all `-m "not gpu"`): brute-force double sum (Eq.
intensity_dble_sum), Bragg-only closed forms of the undisplaced fcc crystal, Friedel symmetry,
Parseval, invariance under supercell translations, the O(n^6) DFT, the Gaussian (Laue)
closed form, the Taylor remainder bound (one order, and per-zone orders against a brute-force
per-atom check and per-order reruns), the 55-FFT count of the fifth-order example,
magnetic projection special cases, the Lanczos m = 2 weights, sub-box closed forms at
n_sb = 1 and an independent pair-sum form, finite differences of the gradient, and the golden
values under tests/golden/.  No function here is "parity unpinned".
"""
from . import core, noise, adjoint  # noqa: F401
from .core import TOTAL, DIFFUSE, C_MAG  # noqa: F401
