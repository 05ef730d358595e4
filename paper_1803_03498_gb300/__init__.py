"""GB300-native HEOM propagator (hierarchical equations of motion, DM-HEOM method).

The compute path is the CUDA library ``libheom`` (C ABI, ``include/heom.h``); ``heom`` is its thin
Python binding.  Importing this package does not load the library: ``heom.load()`` does, and it
raises if the library is missing.
"""
