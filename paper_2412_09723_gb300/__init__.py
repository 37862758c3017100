"""GB300-native differentiable tile-based RGB-D Gaussian rasterizer (MAC-Ego3D,
arXiv 2412.09723): a C-ABI CUDA library for sm_103a and a thin Python binding.

Submodules are imported lazily so that `scenes` (seeded inputs) can be used
without loading the CUDA library.
"""
