"""Posit(32,2) dense linear algebra for GB300 (sm_103a).

Hand-written CUDA kernels behind a C ABI (include/posit_gb300.h); this package
holds the sources (csrc/), the in-tree build (build.py), the ctypes binding
(binding.py) and the seeded input generators (inputs.py).  Importing the
package does not load the CUDA library; the first binding call does, and it
raises if the library has not been built.
"""
__all__ = ["binding", "build", "inputs"]
