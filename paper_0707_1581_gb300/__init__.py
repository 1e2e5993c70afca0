"""GB300 (sm_103a) fluctuating lattice Boltzmann on D3Q19 and D2Q9.

The method is that of Duenweg, Schiller and Ladd (arXiv:0707.1581): the
stream-and-collide update with linear relaxation of every non-conserved mode
and Gaussian noise that satisfies detailed balance.  The CUDA library
(csrc/, C ABI in include/flb.h) does all the work; ``flb`` is its thin ctypes
binding (``HostBuffer``, ``use_torch_allocator`` and the Context methods
included).  ``build`` compiles the library, ``validate`` runs the physics
checks, ``inputs`` makes the seeded synthetic inputs, ``replicas`` and
``tuning`` hold the multi-rank and autotuner-cache helpers.  Importing this
package loads nothing; the library is loaded on the first call.
"""
from . import flb  # noqa: F401

__all__ = ["flb"]
