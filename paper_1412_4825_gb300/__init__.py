"""brng: GB300-native batched RNG for varying-parameter streams (arXiv 1412.4825).

The compute path is the CUDA library ``libbrng.so`` (C ABI declared in
``include/brng.h``); :mod:`paper_1412_4825_gb300.brng` is its ctypes binding.
"""
