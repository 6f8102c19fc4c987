"""GB300-native enumeration of weak pseudo-manifolds over the candidate facets of a mod-2
characteristic map (Choi, Jang, Vallee, arXiv 2301.00806).

Submodules:
  wpm        the binding of libwpm (C ABI in include/wpm.h); loading it builds the library
             if needed and requires a CUDA device to call
  instances  seeded synthetic maps (the benchmark workloads, IDCM orbit representatives)
  build      the nvcc build of libwpm.so

Importing the package loads nothing; the CUDA library is loaded on first use.
"""

__all__ = ["wpm", "instances", "build"]
