"""B300-native batched environment step of Galactic (arXiv 2306.07552).

``gx`` holds the Python binding of the C ABI (include/gx.h); ``inputs`` the
seeded synthetic workloads; ``build`` compiles the CUDA library in-tree.
"""
