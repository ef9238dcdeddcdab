"""GB300-native label propagation (nu-LPA, arXiv 2411.11468): CUDA sweep behind a C ABI.

Submodules:
  lpa       -- ctypes binding of the C-ABI library liblpa.so (the product path)
  graphgen  -- seeded synthetic CSR graph generators (inputs)
  build     -- compiles liblpa.so for sm_103a with nvcc
Importing the package loads nothing; `paper_2411_11468_gb300.lpa` loads the library.
"""
__all__ = ["lpa", "graphgen", "build"]
