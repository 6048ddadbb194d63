"""CPU oracle for the irregular-block sparse LU.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call, link or run anything
here.  The product library never does: it fails loudly when its CUDA build is
missing instead of falling back to CPU code.

* ``oracle.lu``   plain FP64 left-looking Gilbert-Peierls LU without row
  exchanges (C, ``oracle.c``), triangular solves, flop count, backward error.
* ``oracle.plan`` the diagonal block pointer by definition (Algorithm 2's
  result), sampling, the irregular blocking of Algorithm 3 followed step by
  step, regular blocking, and the block task plan of Algorithm 1.

Parity pins (``tests/test_oracle_*.py``) tie every function to something
other than itself: exact recovery of known factors, a library LU on
column-diagonally-dominant dense matrices, brute-force boolean fill, closed
forms of the diagonal block pointer, hand-derived blockings, and brute-force
longest chains of the explicit task graph.  The paper's own blocking example
(Section 4.3, the P0..P5 figure) is an image that is not recoverable, so that
example is "parity unpinned"; every other function has a pin.
"""
from . import lu, plan  # noqa: F401
