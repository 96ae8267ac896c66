"""GB300-native TPC time-frame tracker: cellular-automaton seeding in native
(row, pad, time) coordinates and an FP32 Kalman tracklet fit, as hand-written
sm_103a CUDA behind a C ABI (include/tpcca.h).

``tpcca`` is the ctypes binding; ``_build.build()`` compiles libtpcca.so in tree."""
from . import _build  # noqa: F401

__all__ = ["_build", "tpcca"]
