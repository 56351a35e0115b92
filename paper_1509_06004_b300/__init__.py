"""Batched parametric max-flow / min-cut on 4-connected image grids for B300.

``paper_1509_06004_b300.pmf`` is the ctypes binding of the CUDA library
(``libpmf.so``); ``paper_1509_06004_b300.inputs`` builds seeded synthetic inputs.
Importing the package itself loads nothing.
"""
__all__ = ["inputs", "pmf"]
