"""FP64 CPU oracle for RED accelerated by vector extrapolation (Hong, Romano, Elad,
"Acceleration of RED via Vector Extrapolation").

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct restatement
of the method in float64 NumPy. Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import it. The product path (the CUDA
library and its Python binding) never imports, links or calls anything here, and this
package never imports the product path: the two share no code. Inputs come from the
seeded generator `paper_1805_02158_gb300.synth`, which holds no solver arithmetic.

Modules:
  nlm        -- the denoiser f(x) of Eq. (3): pixelwise non-local means (direct form)
                and a literal per-pixel brute force used to pin it.
  operators  -- the circulant blur H (Fourier diagonalisation), decimation S, adjoints.
  fp         -- one fixed-point step, Eq. (7): Fourier-domain inverse for deblurring,
                conjugate gradients for super-resolution (footnote to Eq. 7).
  ve         -- MPE (Algorithm 1) with MGS QR (Algorithm 2), RRE (Eq. 19) and SVD-MPE.
  red        -- the objective Eq. (4), PSNR, relative change and the cycling driver
                (Algorithm 3), with full cycling or cycling with frozen gamma.
  sd         -- the fixed-step steepest-descent baseline of SD-MPE (Sec. IV), a map of
                one denoiser call per step that the same driver cycles.

Pinning: every function is checked in tests/test_oracle_*.py against facts that do not
come from the oracle itself (brute force, closed forms, dense solves, invariants).
"""
