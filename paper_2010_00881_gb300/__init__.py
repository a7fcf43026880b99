"""GB300-native hierarchical multigrid for the finite cell method.

The compute path is the CUDA library libfcm.so (C ABI in include/fcm.h);
``fcm`` is its ctypes binding and ``build`` compiles it for sm_103a.
"""
from .fcm import (FCM_FP64, FCM_MIXED, FcmError, Solver, load)  # noqa: F401
