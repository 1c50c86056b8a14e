"""GB300-native server hot path of rotation-free HE Conv/FC layers
(arXiv 2409.05205).  The compute path is the CUDA library libhe.so behind the
C ABI in include/he.h; ``paper_2409_05205_gb300.he`` is its ctypes binding.
Importing this package loads nothing; ``he`` loads the library on first use.
"""
