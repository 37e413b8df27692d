"""GB300-native local graph clustering (arXiv:1604.07515).

Submodules:
  ``lgc``     ctypes binding of the CUDA C-ABI library ``liblgc.so``
  ``inputs``  seeded synthetic graphs, seeds and parameters
"""
