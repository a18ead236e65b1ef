"""GB300-native approximate 1-Wasserstein distance between persistence diagrams.

The compute path is the C-ABI library libpdw1.so (hand-written sm_103a CUDA
kernels); `paper_2110_14734_gb300.pdw1` is its thin Python binding.
"""
