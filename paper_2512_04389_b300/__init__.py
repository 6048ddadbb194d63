"""Irregular-block sparse LU for B300 (sm_103a).

``Plan`` (host analysis: symbolic factorization, Algorithm 2 diagonal block
pointer, Algorithm 3 irregular blocking, block task plan), ``Factor`` (GPU
numerical factorization and solves) and ``LUSolve`` (autograd) wrap the C ABI
of ``include/slu.h``.  Importing ``slu`` loads ``libslu_b300.so`` and raises
if it is missing.
"""
__all__ = ["Plan", "Factor", "LUSolve", "lu_solve"]


def __getattr__(name):
    if name in ("Plan", "Factor"):
        from . import slu
        return getattr(slu, name)
    if name in ("LUSolve", "lu_solve"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
