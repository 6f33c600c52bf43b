"""GB300 (sm_103a) latent-rollout library for the WeatherMesh-3 processor.

The compute lives in libwm.so (hand-written CUDA behind the C ABI of
include/wm.h); this package is its thin Python binding.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import WmError, lib, header_functions, make_codec_config, make_config, wm_codec_config, wm_config  # noqa: F401
