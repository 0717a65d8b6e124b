"""GB300-native two-level solver for the 2D high-frequency Lippmann-Schwinger equation.

The compute path lives in a C-ABI CUDA library (`csrc/`, built for sm_103a into
`libls.so`); `binding` is the thin ctypes layer over it.  Importing this package
does not load the library; `binding.load()` does, and raises if it is missing.
"""
