"""GB300 hybrid FEM/FDM solver for conductivity reconstruction (arXiv 1509.01399).

The compute path is the CUDA library libhyb.so (C ABI in include/hyb.h);
``paper_1509_01399_gb300.hyb`` is its Python binding and
``paper_1509_01399_gb300.build`` compiles it in-tree for sm_103a.  Importing
the binding fails when the library has not been built: there is no CPU
fallback.
"""
