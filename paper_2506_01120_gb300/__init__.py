"""GB300 (sm_103a) implementation of the Lie-closure hot path of
"Fast numerical generation of Lie closure" (Iiyama, arXiv 2506.01120):
Algorithm 4, the orthonormalisation method, run in candidate blocks on the GPU.

The package is deliberately thin:

* ``inputs``  -- seeded synthetic generator sets (no closure arithmetic).
* ``binding`` -- ctypes marshalling onto the C ABI of ``liblieclosure.so``
  (``lie_closure``, ``lie_closure_batched`` and their ``*_dev`` forms).
* ``build``   -- nvcc build of the shared library for sm_103a.

Importing the package loads nothing native; ``binding`` loads the library on
first use and raises if it is missing.
"""

__all__ = ["inputs", "binding", "build"]
