"""FP64 CPU oracle for the split-preconditioned fixed-point iteration.

TEST INFRASTRUCTURE, not part of the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import, call or execute anything here.  It shares no code with the CUDA path.

Modules:
  dft         the DFT by its definition (dense matrices, loops)
  usp_oracle  Algorithm 1 with the forward-eliminated operator, FP64
  canon       canonical form (smallest circle, scaling) for Helmholtz and
              diffusion problems
  dense       the operators as dense matrices for brute-force checks
  fno         the Fourier neural operator that proposes a warm start x0:
              forward, hand-derived backward, Adam
  variants    the block forms of Sec. 2.2 (antisymmetrised, for problems
              that are not accretive) and Sec. 3.2 (flux form of diffusion)

Every function pinned by a ``-m "not gpu"`` test; none is marked
"parity unpinned".
"""
