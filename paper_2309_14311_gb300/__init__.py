"""GB300-native (sm_103a) synchronous Nagel-Schreckenberg step on a ring road.

The C ABI lives in ``include/nasch.h``; ``nasch`` is its Python binding.
"""
from . import nasch  # noqa: F401
from .nasch import NaschError, Road, floyd_init, philox_device, slow_threshold  # noqa: F401
