"""GB300-native multi-function direct Monte Carlo integration.

The method is the multi-function mode of ZMCintegral-v5.1 (arXiv 2104.10073):
many integrands with their own form, dimension and box, integrated together by
direct Monte Carlo.  The compute path is the C ABI library ``libzmc.so``
(``include/zmc.h``; CUDA kernels for sm_103a), bound by :mod:`.zmc`.
Importing this package loads nothing; :func:`zmc.lib` loads the library and
raises if it is missing.
"""
