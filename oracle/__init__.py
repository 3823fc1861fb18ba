"""FP64 CPU oracle for the RPA epsilon path (test infrastructure only).

This package is the independent, slow, obviously-correct reference that the
CUDA path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference arm of ``bench.py`` may import it; the library
itself never does, and the oracle never imports the library.

Two tiers, both in complex128 / float64:

* tier 1 (``*_direct``, ``inv_gauss_jordan``): the definitions written out --
  the plane-wave convolution for the matrix elements, explicit sums over
  (v, c) pairs for chi, Gauss-Jordan elimination with partial pivoting for the
  inverse.  Small inputs only.
* tier 2 (``mtxel_fft``, ``chi``, ``inv``): the same quantities through a
  library FFT, a library matrix product and a library inverse, used at the
  larger sizes.

Every function cites the passage of the BerkeleyGW paper (Section
"RPA Dielectric Matrix: epsilon") it follows.  Pins against closed forms,
invariants and brute force live in ``tests/test_oracle_pins.py``.
"""
from .epsilon import (  # noqa: F401
    mtxel_direct, mtxel_fft, band_grids, chi_direct, chi, chi_weights, coulomb,
    eps_sym, eps_asym, inv_gauss_jordan, inv, screened_w, epsinv_sym, solve,
    chi_entries, mtxel_fft_pairs, screened_w_sym, chi_weights_real, frequency_grid, solve_real, realify, sigma_mtxel, density_diag, sigma_cohsex,
)
