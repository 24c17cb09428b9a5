"""Exact string matching on NVIDIA GB300: the SIMD-naive counting search of
Tarhio, Holub and Giaquinta, "Technology Beats Algorithms (in Exact String
Matching)", as a C-ABI CUDA library (include/sm.h) with a thin ctypes binding.

Modules
  sm      binding of the C entry points (sm_histogram, sm_order, sm_count, ...)
  synth   seeded synthetic texts and patterns (input generation only)
  build   in-tree build of the native libraries
"""
