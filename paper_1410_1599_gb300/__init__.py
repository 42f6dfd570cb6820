"""GB300-native multiple-precision GEMM (Simple, Block, Strassen, Winograd)
and LU, after arXiv 1410.1599.

    paper_1410_1599_gb300.binding  ctypes binding of libmpgemm.so (include/mpgemm.h)
    paper_1410_1599_gb300.inputs   seeded synthetic inputs and the interchange format
    paper_1410_1599_gb300.build    builds libmpgemm.so for sm_103a

Importing the package loads nothing; the binding loads the library on first use.
"""
__all__ = ["binding", "inputs", "build"]
