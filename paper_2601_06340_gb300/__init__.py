"""GB300-native two-beam FFT beam-propagation z-march (sm_103a).

The compute path lives in ``csrc/`` (CUDA kernels and a C ABI, declared in
``include/bpm.h``); ``binding`` is a thin ctypes layer over that library and
``inputs`` builds seeded synthetic workloads.  Importing the package loads
nothing; ``binding.load()`` loads the built library and raises if it is
missing.
"""

__all__ = ["binding", "inputs"]
