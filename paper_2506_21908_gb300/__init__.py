"""GB300-native spinor real-time TDDFT propagation step (arXiv 2506.21908).

The compute path is the CUDA library ``libtddft.so`` behind the C ABI declared
in ``include/tddft.h``; this package only marshals arguments to it.
"""
