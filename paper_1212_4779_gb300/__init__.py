"""GB300-native StaticGreedy-DU seed selection (Cheng et al., CIKM'13).

Submodules:
  sg      ctypes binding of the C ABI in include/sg.h (the CUDA library)
  build   compiles csrc/*.cu for sm_103a into _build/libsg.so
  inputs  seeded synthetic graph generators

Importing the package loads nothing; the CUDA library is loaded on first
use of ``paper_1212_4779_gb300.sg``.
"""

__version__ = "0.1.0"
