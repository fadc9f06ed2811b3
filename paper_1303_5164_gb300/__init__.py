"""GB300-native sliced, co-scheduled execution of concurrently submitted kernels
(Kernelet, arXiv 1303.5164): C-ABI library libkernelet.so + thin binding."""
from . import build  # noqa: F401
from .kernelet import *  # noqa: F401,F403
