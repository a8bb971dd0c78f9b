"""GB300 (sm_103a) block-decomposed Huffman coder of Cloud et al.,
"Accelerating Lossless Data Compression with GPUs" (arXiv 1107.1525).

The compute path is libhz.so (CUDA kernels behind the C ABI in include/hz.h);
``paper_1107_1525_gb300.hz`` is its ctypes binding.
"""
