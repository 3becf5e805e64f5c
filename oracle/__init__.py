"""FP64 CPU oracle for the direction-split phi-function action (PHISPLIT).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
this package: only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares no
code with the CUDA library; the only common module is the seeded input generator
``paper_2304_02327_gb300.workloads``, which it does not import either (callers pass
arrays in).

Everything is plain numpy float64, slow and written to be checked against the
paper by eye:

* ``phi``         -- e^X by Pade [13/13] scaling and squaring (Section 3.1, the
                     method named there), and phi_0..phi_lmax of a small matrix
                     from the exponential of a block-augmented matrix.
* ``tucker``      -- mu-mode product (Section 1, eq. (7) taken one direction at
                     a time), Tucker operator (eq. (6)), the split action P_l^(2)
                     of Section 3 (Theorem 1, eq. (14)).
* ``integrators`` -- K u in tensor form, g(u), and the tensor formulations of
                     exponential Euler, ETD2RK, Lawson-Euler and Lawson2b
                     (eq. (17)-(20), Section 3.2).

Each function's pins (what fixes it independently of itself) live in
``tests/test_oracle_*.py``.  Parity of every function here is pinned; none is
"parity unpinned".
"""
from .phi import expm_pade13, phi_matrices, PADE13_THETA  # noqa: F401
from .tucker import mode_product, tucker, phisplit_apply  # noqa: F401
from .integrators import (kron_apply, g_eval, step, step_at, integrate,  # noqa: F401
                          rel_err_inf, rel_err_fro, OracleProblem)
