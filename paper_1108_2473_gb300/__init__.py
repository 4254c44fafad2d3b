"""GB300 (sm_103a) library for the hot path of disconnected fermion loops (arXiv:1108.2473).

The computation lives in liblqcd.so (CUDA, built in-tree by ``build_lib.build()``)
behind the C ABI of ``include/lqcd.h``; ``lqcd`` is its ctypes binding.
"""
from . import lqcd  # noqa: F401
from .lqcd import *  # noqa: F401,F403

__all__ = [n for n in dir(lqcd) if n.startswith(("lqcd_", "LQCD_"))] + ["LqcdError", "solver_params"]
