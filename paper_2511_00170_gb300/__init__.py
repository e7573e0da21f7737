"""GB300 in-silico PCR engine: the AmpliconHunter2 hot path (arXiv 2511.00170) as sm_103a CUDA
kernels behind the C ABI in ``include/ah.h``; :mod:`.ah` is its ctypes binding and
:mod:`.pipeline` runs the whole path through it."""
