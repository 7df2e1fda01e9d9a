"""FP64 CPU oracle for CUBE's compressed-store particle-mesh step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline / reference leg may import it; the library
(paper_1712_06121_gb300) never does, and this package imports nothing from it.

It follows the paper step by step in FP64 (numpy), with numpy's FFT, stable
argsort and bincount as library steps:
  codec.py   Eqs. chi / x (position codes), Eqs. nu / v (velocity codes),
             Section 2.1-2.2
  layout.py  cell-ordered storage (Section 2.1, 2.3.1): counts -> offsets,
             storage order of coarse cells
  mesh.py    CIC deposit, Poisson solve with Green's function and CIC
             deconvolution, 4th-order finite-difference gradient, CIC gather,
             power spectrum (Section 3.2, Eq. cps)
  cosmo.py   expansion rate, kick/drift factors, linear momentum growth
  pm.py      the compressed store and one KD step (Fig. update_xp /
             update_vp, Section 2.3.3), plus an uncompressed FP64 mode
  pp.py      brute-force pairwise force (used only to pin mesh.py)

Where the paper leaves a passage open, the function that depends on it
states the reading it takes.
"""
from . import codec, layout, mesh, cosmo, pm, pp  # noqa: F401
