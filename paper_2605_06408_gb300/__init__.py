"""GB300-native construction of 3D Voronoi and power diagrams.

The compute path is a C-ABI CUDA library (``libvd.so``, declared in
``include/vd.h``); :mod:`paper_2605_06408_gb300.vd` is its thin binding.
Importing the package does not load the library.
"""
