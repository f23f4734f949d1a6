"""FP64 oracle for the RMRT-LB step (test infrastructure only; see rmrt.py)."""
from .rmrt import *  # noqa: F401,F403
