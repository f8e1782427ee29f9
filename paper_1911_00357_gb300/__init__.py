"""GB300-native (sm_103a) DD-PPO rollout-then-update hot path (arXiv:1911.00357).

The compute lives in ``_build/libddppo.so`` (CUDA kernels behind the C ABI of
``include/ddppo.h``); ``binding`` is a thin ctypes layer with the same names,
``worker`` allocates rollout buffers with torch and drives the loop.
"""
from . import binding  # noqa: F401
from .presets import make_config, PRESETS  # noqa: F401
