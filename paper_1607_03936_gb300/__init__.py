"""GB300-native w-BFBT Stokes solver (Rudi, Stadler & Ghattas, arXiv 1607.03936).

The compute path is the CUDA library libwbfbt.so (C ABI in include/wbfbt.h);
`paper_1607_03936_gb300.wbfbt` is its thin Python binding and
`paper_1607_03936_gb300.inputs` draws the seeded synthetic inputs.  Importing
the package itself loads neither torch nor the library.
"""
