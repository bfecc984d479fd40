"""FP64 CPU oracle for KK beamforming and CPWC DAS.

TEST INFRASTRUCTURE -- not part of the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) may import, call, link or run anything in this
package.  The product library never routes through it; the oracle shares no
code, tables or helpers with the CUDA path.  Its only shared dependency is the
seeded input generator ``kksynth``, which holds none of the method's
arithmetic.

Contents (each function cites the passage of Khetan & Mertz, "Far-field
compressive ultrasound beamforming", that it follows):

* ``schemes``  -- receive-angle schemes and pair sets (Section II-C, Eq.
  (uniform); Section II-D, Eq. (confocal); hybrid groups, Eqs.
  (coherent)/(incoherent)).
* ``kk``       -- analytic signal (Section II-F), far-field decomposition
  (Eq. (compression) via the Fourier shift theorem, Section II-F), KK image
  formation (Eq. (KK)), DAS (Eq. (DAS)), compounding.
* ``kk_oracle.c`` -- the pixel x pair loops in plain FP64 C.
* ``volume``   -- volumetric KK and DAS with a 2D (matrix) array: plane
  waves in three dimensions, the extension Section IV names.
* ``quality``  -- image-quality measures the paper judges images by: gCNR of
  an inclusion against a background region and half-amplitude widths of
  point targets (Section III, Figs. 4 and 5).

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants, brute force or the paper's stated properties; see the test
docstrings for which mistake each pin would catch.
"""
from . import schemes, kk, quality, volume  # noqa: F401
