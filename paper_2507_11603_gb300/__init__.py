"""GB300-native resonant-line Monte Carlo hot path (THOR, arXiv:2507.11603).

libthor.so (CUDA, sm_103a) implements the Lyman-alpha photon-packet loop and the
Lyman-alpha forest ray-march behind the C ABI in include/thor.h; ``thor`` is the
ctypes binding; ``synth`` holds the seeded synthetic input generators.
"""
from . import _build  # noqa: F401
from .thor import Context, Server, ThorError, line_params, load  # noqa: F401

__all__ = ["Context", "Server", "ThorError", "line_params", "load"]
