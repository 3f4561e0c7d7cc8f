"""CPU oracle for the SLSE-FRS hot path: plain, slow, FP64, written from the paper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA library never calls it, and it shares no code with the CUDA path: the
counter-based generator, the Hadamard transform, the sampling, the QR and the
M-IHS iteration are all written here a second time from their published
definitions.

Paper: "Sequential Least-Squares Estimators with Fast Randomized Sketching for
Linear Statistical Models" (arXiv 2509.06856).

Modules
-------
philox  - Philox4x32-10 (Salmon et al., SC'11), the generator both sides use.
sketch  - random draws D, P, sigma; Walsh-Hadamard transform; SRHT (Sec. 3).
countsketch - the CountSketch family (Sec. 2; the SLSE-FRS-CS experiment of Sec. 5).
adjoint - gradients through the least-squares estimate (dense formulas, finite differences).
fp8     - E4M3 values with 32-element power-of-two block scales (OCP FP8 / MX definitions).
linalg  - Householder QR, OLS via QR (Sec. 1), triangular solves.
slse    - schedules, a_i bound (Thm 4.3), gradient, M-IHS update, Algorithm 2.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` except the stage-1 iterate values for schedules
with m_1 <= r, which the paper's theorems do not cover ("parity unpinned" for
those intermediate values; the final estimate is pinned to OLS).
"""
from . import philox, sketch, countsketch, linalg, slse, adjoint, fp8  # noqa: F401
