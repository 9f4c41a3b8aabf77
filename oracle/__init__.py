"""Plain, slow FP64 CPU oracle for the spinor real-time propagation step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.  The
CUDA library never calls it, shares no code, table or constant generator with
it, and fails loudly when its own extension is missing.

Every function cites the passage of arXiv 2506.21908 it follows.  Where the
paper is silent (propagator, projector radial shapes, XC parameterisation,
thresholds) the oracle takes one stated reading; the readings are listed in
the module docstrings and in the design notes.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, brute force or invariants (tests/test_oracle_*.py).  The
absolute values of n(t), m(t) in the synthetic systems are not pinned beyond
those invariants ("parity unpinned" for physical magnitudes: the paper's own
systems need pseudopotential files that are not available).
"""
from .tddft import System, Oracle  # noqa: F401
