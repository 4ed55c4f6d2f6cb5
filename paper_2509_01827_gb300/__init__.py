"""GB300-native explicit MCT-2D-CEM time step (arXiv 2509.01827).

``paper_2509_01827_gb300.cem`` is the thin ctypes binding of the CUDA C-ABI
library ``libcem.so`` (declared in ``include/cem.h``); ``inputs`` holds the
seeded problem generators.  Importing the package loads nothing native.
"""
