"""GB300-native step-off TEM forward model (shared-pole rational approximant + batched shifted COCG).

The compute path lives in the C-ABI shared library built from ``csrc/`` (see
``include/tem.h``); ``tem`` is its thin ctypes binding.  Importing this package
does not load the library; ``tem.lib()`` does, and fails loudly if it is missing.
"""
