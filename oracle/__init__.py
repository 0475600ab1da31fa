"""FP64 CPU oracle for separable W-projection gridding (Merry 2015).

TEST INFRASTRUCTURE.  This package is the plain, slow reference the CUDA path
is checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path never does.
It shares no code, headers or tables with the CUDA library and never takes an
input or expected value from it.

Contents (each function cites the passage it follows):
  * ``sepw_oracle``  taper, 1-D taps (Eq. gt), exact 2-D kernel table, cell /
                     plane location, brute-force dirty image and prediction
                     (Eq. dirty and the prediction integral, Sec. 2), the image
                     step with grid correction, hybrid W stacking (Sec. 4.3),
                     and the analysis formulas of Secs. 2-4 and Appendix A;
  * ``sepw_oracle.c`` plain C FP64 loops: separable gridder (Sec. 5), its
                     adjoint degridder, and the exact 2-D kernel gridder.

Parity status: every function is pinned by a ``-m "not gpu"`` test except the
accuracy of truncated-support gridding against the direct sum, which the paper
does not bound ("parity unpinned": it is reported as a measured number only).
"""
from .sepw_oracle import *  # noqa: F401,F403
