"""GB300-native Icarus MHD update (arXiv 2211.12867): CUDA kernels for sm_103a
behind a C ABI (``libicarus.so``), with a thin ctypes binding."""
