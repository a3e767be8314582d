"""GB300-native (sm_103a) Axilrod-Teller-Muto three-body forces over linked-cell
triplets, next to Lennard-Jones pair forces (arXiv 2510.21230).

The compute path is the CUDA library ``libatm3.so`` behind the C ABI of
``include/atm3.h``; ``atm3`` is its ctypes binding, ``synth`` draws the seeded
synthetic inputs, ``build`` compiles the library in-tree.
"""
__all__ = ["atm3", "synth", "build"]
