"""GB300 resolution-of-the-identity Coulomb/exchange engine for PNOF7 (arXiv 2012.15662).

The compute path is the CUDA shared library `libdonof_ri.so` built from
`csrc/` for sm_103a; `binding` wraps its C ABI (`include/donof_ri.h`) with
ctypes.  Importing this package loads nothing; `binding.load()` (called by
every binding function) raises if the library is missing -- there is no CPU
fallback.
"""
__all__ = ["binding", "build"]
