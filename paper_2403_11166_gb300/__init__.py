"""GB300-native (sm_103a) hot path of Pencil's homomorphic linear layers.

Import `paper_2403_11166_gb300.he` for the C-ABI binding; it loads the CUDA
library built by `paper_2403_11166_gb300.build` and raises if it is missing.
"""
__version__ = "0.1.0"
