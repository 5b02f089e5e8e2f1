"""GB300 theta-method library for eddy-current transients (arXiv 2407.11993).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/eddy_theta.h``); ``eddy`` is its ctypes binding.
"""
