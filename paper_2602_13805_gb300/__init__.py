"""GB300 (sm_103a) implementation of the PDF inverse-scattering solver's hot path.

The compute lives in the CUDA library libpdf.so behind the C ABI of include/pdf.h;
`paper_2602_13805_gb300.pdf` is its thin Python binding.  Importing this package
loads nothing; the first library call does, and fails loudly if libpdf.so is missing.
"""
from . import pdf  # noqa: F401
