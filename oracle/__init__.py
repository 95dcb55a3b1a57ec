"""Plain FP64 CPU oracle for the periodic piezoelectric cell problem.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
reference that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm
may import it; the library never does, and the oracle imports nothing from the
library.  The two share only the seeded input generators in ``cellgen``.

What it computes (paper: Wegert, Roberts & Challis, "Level set-based inverse
homogenisation of three-dimensional piezoelectric materials", arXiv 2410.03148):

* material tensors and their nondimensionalisation (§2.2, following Cao &
  Neytcheva) -- ``material``;
* the Q1 hexahedral element matrix of the coupled elasticity/electrostatics
  bilinear form, the nine affine macroscopic loads, periodic sparse assembly of
  the symmetric indefinite block system of Eq. (sym-piezo), and its direct
  solution -- ``fem``;
* the homogenised tensors of Eqs. (hom_C), (hom_e), (hom_kappa), both in the
  paper's linear form and in the equivalent energy form -- ``fem``;
* the smoothed-boundary ersatz material of §2.6 -- ``ersatz``;
* the figures of merit of §2.3 (d_h, B_Voigt, B_Reuss) -- ``figures``;
* element-wise sensitivities of the homogenised tensors and a finite
  difference checker -- ``sensitivity``;
* the exact homogenisation of a layered (laminate) cell -- ``laminate``;
* a brute-force dense solver and brute-force quadrature -- ``dense``.

Every function is pinned by a ``-m "not gpu"`` test against a closed form, an
invariant or brute force (see tests/test_oracle_*.py).
"""
