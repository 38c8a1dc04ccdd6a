"""FP64 CPU oracle of the PDF (physics-driven Fourier-spectral) solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the paper's forward model, loss and gradient in
float64 NumPy/SciPy.  It exists so the CUDA path can be checked against it.
Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import it; the product path (the C-ABI library and its Python binding) never
does, and shares no code with it.

Modules
  problem   the problem description (grid, wavenumber, antennas, Fourier truncation)
  green     Richmond pulse-basis operators G_D (dense and FFT-applied), G_S, E_inc  (Eq. 1-4)
  forward   the forward scattering solve (Eq. 3-5) used to synthesise measured data
  mie       Bessel-series scattered field of a homogeneous cylinder (independent pin)
  fbe       truncated Fourier basis expansion J = F*_T(alpha), alpha = F_T(J)      (Eq. 9)
  loss      the composite loss L and its hand-derived gradient dL/d alpha      (Eq. 6, 7, 13-19)
  cco       contrast-compensated operator (Eq. 10, 11) with the self-guided filter, and its adjoint
  solve     BP + one-step CSI initialisation (Eq. 12), Adam loop, final CCO, RelErr
  mlp       FP64 reference of the warm-start network forward/backward

Parity status of each function is stated in its docstring ("pinned by ..." or
"parity unpinned").
"""
