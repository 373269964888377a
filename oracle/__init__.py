"""Plain FP64 CPU oracle for RTCUR. Test infrastructure only (see rtcur_oracle.py)."""
from .rtcur_oracle import *  # noqa: F401,F403
from . import rtcur_adjoint  # noqa: F401
