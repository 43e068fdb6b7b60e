"""GB300-native Super Bloom filter: sequence-native insert and query of DNA k-mers.

The compute path is the CUDA library ``libsbf.so`` (C ABI in ``include/sbf.h``),
bound here with ctypes; PyTorch only supplies device memory and streams.
"""
