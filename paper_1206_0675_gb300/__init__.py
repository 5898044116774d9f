"""lgf: Fourier-accelerated steepest-descent Landau gauge fixing on GB300.

The compute path is the C-ABI library ``liblgf.so`` (CUDA, sm_103a); ``lgf``
holds its ctypes binding.  Importing this package does not load the library;
``paper_1206_0675_gb300.lgf`` does, and fails loudly if it has not been built.
"""
