"""GB300-native live ePIE engine (arxiv 2308.10674, "Live Iterative Ptychography").

The reconstruction runs in libepie.so (hand-written sm_103a CUDA behind the C
ABI of include/epie.h); this package only marshals arguments to it.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import Engine, EpieError, lib  # noqa: F401
