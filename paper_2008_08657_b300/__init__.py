"""B300-native engine for batches of group-by aggregates over joins (LMFAO, arXiv 2008.08657).

Submodules: ``lmfao`` (ctypes binding of ``include/lmfao.h``), ``workloads`` (seeded
synthetic inputs), ``build`` (compiles ``liblmfao.so`` for sm_103a). Importing the package
loads nothing.
"""
