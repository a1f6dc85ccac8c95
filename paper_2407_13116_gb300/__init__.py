"""libk2svd: batched SVD of real 2x2 matrices by the enhanced Kogbetliantz method
(arXiv 2407.13116) on GB300 (sm_103a).

The compute path is the CUDA library ``csrc/libk2svd.so`` behind the C ABI declared
in ``include/k2svd.h``; ``k2svd`` is its thin Python binding (argument marshalling
only).  Importing this package does not load the library; ``k2svd`` does, and fails
loudly when it is missing.
"""
