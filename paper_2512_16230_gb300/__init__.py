"""GB300-native MRT lattice Boltzmann on multispeed rectangular lattices (arXiv 2512.16230).

The compute path is the C-ABI CUDA library built from ``csrc/`` (declared in
``include/lbm_mrt.h``); ``lbm`` is its thin ctypes binding. Importing this package does not load
the library, so the input generators can be used on machines without a GPU; every call into
``lbm`` raises if the library is missing.
"""
__all__ = ["lbm", "inputs", "workloads", "build"]
