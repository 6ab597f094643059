"""GB300-native projective-dynamics cloth stepper (arXiv 2403.19272).

The solve runs in libpdcloth.so (CUDA, sm_103a) behind the C ABI declared in
include/pdcloth.h; ``pdcloth`` is its ctypes binding and ``build`` compiles
it in-tree.
"""
__all__ = ["build", "pdcloth"]
