"""FP64 CPU oracle for the IMEX-TR hot path (test infrastructure).

This package is a plain, slow, obviously correct restatement of the paper's method
(arXiv 2603.03933: discretised Landau-Brazovskii energy, §2; IMEX trust-region
method, §3) used only to check the CUDA path.  It shares no code with the CUDA
library and imports nothing from it.  Only the test suite, the smoke check of
`__graft_entry__` and the CPU-baseline / reference arm of `bench.py` may import it;
the product path never calls it.

Modules and what pins them (tests/test_oracle_*.py):
  fft          own radix-2 DFT   <- direct O(M^2) DFT, numpy.fft, Parseval
  lb           energy/grad/Hv     <- closed-form lamellar energies, the paper's
                                     Fourier-space convolution sums evaluated by
                                     enumeration, Richardson-exact finite
                                     differences (E is quartic, g cubic along lines)
  subproblem   Algorithm 3        <- exact dense More-Sorensen minimiser, the
                                     optimality conditions, monotone descent
  trust_region Algorithms 1, 2    <- second-order stationarity at exit (dense
                                     eigenvalues), PCG vs dense solve
  eig          lambda_min         <- dense eigendecomposition, closed form at psi = 0
  first_order  semi-implicit      <- closed-form step on a single cosine mode,
               gradient flow         monotone energy decrease, fixed points = zeros of g
"""
