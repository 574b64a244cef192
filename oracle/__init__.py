"""CPU oracle for guaranteed upper-lower bounds by the FFT-based Galerkin method.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or execute
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares no
code with the CUDA library; the only common dependency is the geometry-only
``microstructures`` package that describes the synthetic inputs.

Everything here is plain NumPy/SciPy in float64/complex128, written from
J. Vondrejc, J. Zeman, I. Marek, "Guaranteed upper-lower bounds on homogenized
properties by FFT-based Galerkin method":

  fourier.py  closed-form Fourier coefficients of the matrix-inclusion coefficient
              (Eq. A_with_inclusions, Lemma bounds_for_matrix-inclusion, Remark
              "inclusion"; the ball/disk transforms are the textbook transforms of
              the indicator, the paper only cites them), the projections
              Gamma^E / Gamma^J (Def. projection).
  dense.py    O1: the Galerkin problem written out as its definition: the dense
              Fourier-Galerkin matrix of Lemma Ga_full, the constrained minimum
              solved by LU, the bound energies of Def. upper_lower_bounds.
  matfree.py  O2: the paper's algorithm steps with the exact double-grid
              quadrature of Lemma double-grid inside the matvec: zero-pad to
              the 2N-1 grid, naive (matrix) DFTs, pointwise coefficient, truncation,
              projection, conjugate gradients (Sec. 6.1) and the double-grid energy.
  bounds.py   upper / lower / mean / guaranteed error (Eq. approx_homog_with_error).
  gani.py     GaNi (Def. GaNi, Cor. FD_GaNi): the coefficient sampled at the grid
              points, the grid-quadrature Galerkin matrix, its minimisers, the GaNi
              homogenized matrices and the bounds of the paper's algorithm (the
              minimisers in the exactly integrated forms, Eq. GaNi_bounds).
  fno.py      the learned warm start's Fourier-layer network in PyTorch float64.
  image.py    pixel-image values, with the paper's optional 4/2/1 local average
              (Sec. 7.3) written as circulant-matrix products.

Every function is pinned by ``tests/test_oracle_pins.py``,
``tests/test_oracle_gani_pins.py`` and ``tests/test_oracle_fno_pins.py`` against facts the
paper and the mathematics fix (Voigt-Reuss, laminates, the 2D rotation identity,
monotonicity in N, brute-force quadrature, odd-grid GaNi duality, ...).
"""
from .fourier import (coefficient_hat_at, coefficient_hat_grid, freqs, projection,
                      topology_hat_at, phase_inverse)
from .dense import dense_bounds, dense_energy_matrix, dense_fields
from .matfree import (MatFreeOperator, cg_solve, matfree_bounds, matvec_sampled)
from .bounds import assemble_bounds
from .image import image_values, smoothed_image, smoothing_matrix

__all__ = [
    "coefficient_hat_at", "coefficient_hat_grid", "freqs", "projection", "topology_hat_at",
    "phase_inverse", "dense_bounds", "dense_energy_matrix", "dense_fields", "MatFreeOperator",
    "cg_solve", "matfree_bounds", "matvec_sampled", "assemble_bounds", "image_values",
    "smoothed_image", "smoothing_matrix",
]
