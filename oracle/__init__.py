"""Float64 CPU oracle of the 3DGS training step.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import, build or call anything in this package.  It
shares no code, header, table or constant with the CUDA path; both sides only
share the seeded input generators in ``synth``.

Modules:
  preprocess  per-Gaussian projection + SH colour (+ autograd backward)
  render      per-pixel blend and per-pixel backward (C, OpenMP)
  loss        L1 and SSIM loss with their image gradients
  adam        Adam update
  binning     brute-force tile sets and stable sort definitions
  step        one whole training step composed from the above
  densify     score-guided densification and pruning (Sec. 3.2)
  ng          neural-Gaussian decoder (Sec. 2.3)
  pose        global pose correction: its gradient and update (Sec. 2.5)
"""
