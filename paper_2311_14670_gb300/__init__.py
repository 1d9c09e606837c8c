"""GB300-native spin spherical-harmonic and Wigner transforms (Price & McEwen, arXiv:2311.14670).

The compute path is libs2gb.so (hand-written CUDA for sm_103a, C ABI in include/s2gb.h); this
package only marshals arguments.  Importing it does not load the library; the first plan does,
and raises if the library was not built.
"""
from .transforms import Plan, forward, inverse  # noqa: F401

__all__ = ["Plan", "forward", "inverse"]
