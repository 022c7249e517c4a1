"""GB300-native IE forward model with domain decomposition (Saputera et al., arXiv 2306.17537).

The compute path is the C-ABI library ``libie_gb300.so`` (hand-written sm_103a CUDA, declared in
``include/ie.h``); ``paper_2306_17537_gb300.ie`` is its thin ctypes binding. Importing this package
does not load the library; importing ``.ie`` does, and fails loudly if it has not been built.
"""
